"""Host-only audit of the step kernels' shared-memory plans (no GPU): the
plans of the benchmarked batches, the uneven batch of the GPU tests (1,500
envs, seed 3) and of the benchmark (65,536 envs), and edge shapes, each alone
and in CTA groups, with every flag combination, checked against sizes
recomputed from the env parameters (`tests/plan_audit.cu`)."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

from paper_2604_27162_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2604_27162_gb300", "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def audit(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("plan_audit") / "plan_audit")
    subprocess.run([nvcc, "-O1", "-std=c++17", "-I", CSRC, "-I", INC, os.path.join(HERE, "plan_audit.cu"), "-o", exe],
                   check=True, capture_output=True, timeout=600)
    return exe


def _line(d):
    return "%d %d %d %d %d %d" % (d["side"], d["n_agents"], d["n_seekers"], d["r_seek"], d["r_hide"],
                                  d.get("obs_teams", 3))


def _run(exe, descs):
    out = subprocess.run([exe], input="\n".join(_line(d) for d in descs) + "\n", capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0 and out.stdout.startswith("OK"), out.stdout[-2000:]
    return int(out.stdout.split()[1])


def test_plans_of_the_benchmarked_batches(audit):
    descs = [W.ten1k()["descs"][0]] * 8 + [W.single1k()["descs"][0]] * 8 + [W.plain16()["descs"][0]] * 4
    assert _run(audit, descs) > 0


def test_plans_of_the_uneven_batches(audit):
    """The uneven batch of the GPU tests and the first 4,096 envs of the
    benchmark's, sorted by shape as the grouping packs them."""
    for descs in (W.uneven_descs(1500, 3), W.uneven_descs(65536, 3)[:4096]):
        key = lambda d: (d["n_agents"], d["r_seek"], d["r_hide"], d["side"] + 8 > 64, d["side"] > 32)
        assert _run(audit, sorted(descs, key=key)) > 0


def test_plans_of_edge_shapes(audit):
    """Sides 2-64, 1-32 agents, radii 0-4, every observing-team setting with
    and without line of sight or decentralized planes."""
    descs = []
    for side in (2, 8, 31, 32, 33, 56, 57, 64):
        for A in (1, 2, 5, 16, 17, 32):
            if A > side * side:
                continue
            for r in (0, 1, 3, 4):
                for teams in (1, 2, 3, 3 | 4, 2 | 4, 3 | 8, 0):
                    descs += [W.env_desc(side, A, (A + 1) // 2, r, max(0, r - 1), 10, "0.1", teams)] * 3
    assert _run(audit, descs) > 0
