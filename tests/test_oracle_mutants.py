"""Mutation test of the oracle's pins (CPU only).

Each mutant plants one plausible mistake in a copy of the oracle's C source
(a dropped term, a wrong sign or index, a transposed operand; a few need two edits to stay consistent), builds it with
gcc in a temporary directory and runs the pin battery against it in a child
process.  Every mutant must fail at least one pin; the unmodified oracle must
pass them all.  The mistakes are planted in the oracle, on the CPU only.
"""
from __future__ import annotations

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hase_oracle.c")

MUTANTS = [
    ("philox multipliers transposed", "uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;",
     "uint64_t p0 = (uint64_t)PHILOX_M1 * (uint64_t)c0;"),
    ("philox hi/lo transposed", "uint32_t n1 = (uint32_t)p1;", "uint32_t n1 = (uint32_t)(p1 >> 32);"),
    ("philox key bump dropped", "k1 += PHILOX_W1;", "k1 += 0u;"),
    ("philox xor term dropped", "^ c3 ^ k1;", "^ k1;"),
    ("action word index", "return mulhi32(out[t & 3u], 5u);", "return mulhi32(out[0], 5u);"),
    ("action range", "return mulhi32(out[t & 3u], 5u);", "return mulhi32(out[t & 3u], 4u);"),
    ("action counter transposed", "philox_words(seed, (uint32_t)(t >> 2), agent, env_id, 0u, out);",
     "philox_words(seed, (uint32_t)(t >> 2), env_id, agent, 0u, out);"),
    ("north sign", "static const int32_t DY[5] = {0, -1, 1, 0, 0};",
     "static const int32_t DY[5] = {0, 1, -1, 0, 0};"),
    ("occupancy check dropped", "if (x[b] == tx[a] && y[b] == ty[a]) ok[a] = 0;", ";"),
    ("obstacle check dropped", "if (ok[a] && grid[(size_t)ty[a] * S + (size_t)tx[a]] != 0) ok[a] = 0;",
     ";"),
    ("highest index wins", "for (uint32_t b = 0; b < a && moves; ++b) {",
     "for (uint32_t b = a + 1; b < A && moves; ++b) {"),
    ("reward strict distance", "if (cheb <= (int32_t)r_seek) seen = 1;",
     "if (cheb < (int32_t)r_seek) seen = 1;"),
    ("reward hider sign", "rew[h] = seen ? -1 : 0;", "rew[h] = seen ? 1 : 0;"),
    ("obs index transposed", "uint32_t k = (uint32_t)((dy + R) * D + (dx + R));",
     "uint32_t k = (uint32_t)((dx + R) * D + (dy + R));"),
    ("obs out-of-bounds not obstacle", "                out[0 * W + word] |= bit;\n                continue;",
     "                continue;"),
    ("obs self not excluded", "                if (b == a) continue;\n", ""),
    ("obs planes swapped", "                    out[1 * W + word] |= bit;\n                else\n                    out[2 * W + word] |= bit;",
     "                    out[2 * W + word] |= bit;\n                else\n                    out[1 * W + word] |= bit;"),
    ("done one step early", "if (w->ep_t[e] == p->cap) {", "if (w->ep_t[e] + 1 == p->cap) {"),
    ("reset keeps positions", "            w->x[base + a] = w->sx[base + a];\n            w->y[base + a] = w->sy[base + a];\n        }\n    }\n    if (rew)",
     "        }\n    }\n    if (rew)"),
    ("start cells not forced free", "for (uint32_t a = 0; a < p->n_agents; ++a) g[cells[a]] = 0;", ";"),
    ("start duplicates allowed", "if (cells[b] == cell) dup = 1;", ";"),
    ("obstacle word index", "g[c] = out[c % 4u] < p->density_thr ? 1 : 0;",
     "g[c] = out[0] < p->density_thr ? 1 : 0;"),
    ("line of sight rounds down", "return p >= 0 ? (2 * p + n) / (2 * n) : -((-2 * p + n) / (2 * n));",
     "return p >= 0 ? p / n : -((-p) / n);"),
    ("central ignores observing teams", "                if (!((obs_teams >> team) & 1u)) continue;\n                const int32_t r = (int32_t)(team ? r_hide : r_seek);",
     "                const int32_t r = (int32_t)(team ? r_hide : r_seek);"),
    ("desync offset word", "return mulhi32(out[0], w->env[e].cap);", "return mulhi32(out[1], w->env[e].cap);"),
    ("pre-steps from the step stream", "philox_words(seed, tau >> 2, agent, env_id, 4u, out);",
     "philox_words(seed, tau >> 2, agent, env_id, 0u, out);"),
    ("one pre-step fewer", "for (uint32_t tau = 0; tau < n; ++tau) {", "for (uint32_t tau = 1; tau < n; ++tau) {"),
    ("pre-step word", "return mulhi32(out[tau & 3u], 5u);", "return mulhi32(out[(tau + 1u) & 3u], 5u);"),
    ("no pre-steps", "if (w->desync) prestep_env(w, e, w->ep_t[e]);", "if (w->desync) prestep_env(w, e, 0u);"),
    ("fog map kept across episodes", "const uint8_t before = start ? 0 : d[c];", "const uint8_t before = d[c];"),
    ("fog fresh is the whole map", "f[c] = (uint8_t)(seen && !before);", "f[c] = (uint8_t)(before | seen);"),
    ("fog per-agent unit ignores its agent", "const uint32_t mine = !per_agent || k == u;",
     "const uint32_t mine = 1;"),
    ("fog not updated on steps", "    if (w->fog) fog_env(w, e, d != 0);\n", "\n"),
    ("true state x and y transposed", "cells[i] = (uint16_t)((uint32_t)w->x[i] | ((uint32_t)w->y[i] << 6));",
     "cells[i] = (uint16_t)((uint32_t)w->y[i] | ((uint32_t)w->x[i] << 6));"),
    # a consistent transposition: agents start at (cell / S, cell % S) and
    # that cell is the one forced free, so every invariant still holds
    ("start x and y transposed", [
        ("w->sx[base + a] = (int32_t)(cells[a] % S);\n        w->sy[base + a] = (int32_t)(cells[a] / S);",
         "w->sx[base + a] = (int32_t)(cells[a] / S);\n        w->sy[base + a] = (int32_t)(cells[a] % S);"),
        ("for (uint32_t a = 0; a < p->n_agents; ++a) g[cells[a]] = 0;",
         "for (uint32_t a = 0; a < p->n_agents; ++a) g[(cells[a] % S) * S + cells[a] / S] = 0;")]),
    ("obstacle counter c instead of c / 4", "philox_words(w->seed, c / 4u, 0u, env_id, 1u, out);",
     "philox_words(w->seed, c, 0u, env_id, 1u, out);"),
    ("splitmix64 first shift", "z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;",
     "z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;"),
]


def _edits(m):
    """(old, new) replacements of a mutant: one pair, or a list of pairs."""
    return m[1] if isinstance(m[1], list) else [(m[1], m[2])]


@pytest.fixture(scope="module")
def aten_driver(tmp_path_factory):
    import torch

    from tests.test_oracle_pins import _ATEN_DRIVER

    d = tmp_path_factory.mktemp("aten")
    src = d / "drv.cpp"
    exe = d / "drv"
    src.write_text(_ATEN_DRIVER)
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-I", inc, str(src), "-o", str(exe)])
    return str(exe)


def _build(src_text, d):
    c = d / "m.c"
    so = d / "libm.so"
    c.write_text(src_text)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-I",
                           os.path.join(ROOT, "oracle"), str(c), "-o", str(so)])
    return str(so)


def _battery(so, drv):
    out = subprocess.run([sys.executable, "-m", "tests.pin_battery", so, drv], cwd=ROOT,
                         capture_output=True, text=True, timeout=120)
    if out.returncode != 0:
        return ["crashed"]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_unmodified_oracle_passes_battery(tmp_path, aten_driver):
    so = _build(open(SRC).read(), tmp_path)
    assert _battery(so, aten_driver) == []


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(mutant, tmp_path, aten_driver):
    name = mutant[0]
    text = open(SRC).read()
    for old, new in _edits(mutant):
        assert text.count(old) == 1, name
        text = text.replace(old, new)
    so = _build(text, tmp_path)
    failed = _battery(so, aten_driver)
    assert failed, "mutant not caught: " + name
