"""hase_digest_noalloc (the digest with the library's fixed scratch) against
hase_digest (the handle's scratch), two calls in a row, on the GPU.  Collected
last so that it runs alone and after every other test."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2604_27162_gb300 import hase
from paper_2604_27162_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _both(eng, n_steps):
    import torch

    a = torch.zeros(4, dtype=torch.int64, device="cuda")
    b = torch.zeros(4, dtype=torch.int64, device="cuda")
    ra = torch.zeros(eng.layout["agents"], dtype=torch.int64, device="cuda")
    rb = torch.full((eng.layout["agents"],), -7, dtype=torch.int64, device="cuda")
    hase.hase_digest(eng.h, n_steps, a.data_ptr(), ra.data_ptr(), eng.stream)
    hase.hase_digest_noalloc(eng.h, n_steps, b.data_ptr(), rb.data_ptr(), eng.stream)
    torch.cuda.synchronize()
    return a.cpu().numpy(), b.cpu().numpy(), ra.cpu().numpy(), rb.cpu().numpy()


@pytest.mark.parametrize("case", ["ten", "uneven"])
def test_noalloc_digest_equals_digest_twice(case):
    if case == "ten":
        c = W.ten1k()
        eng = hase.Engine(200, c["seed"], [dict(c["descs"][0], cap=31)], ring_steps=96)
    else:
        eng = hase.Engine(300, 3, W.uneven_descs(300, 4), ring_steps=64)
    eng.step(70)
    first = _both(eng, 60)
    second = _both(eng, 60)  # a second call in a row reuses the same scratch
    for x, y in zip(first, second):
        assert np.array_equal(x, y)
    a, b, ra, rb = first
    assert np.array_equal(a, b)
    assert np.array_equal(ra, rb)
    assert a[0] != 0 and a[3] == 0  # a real digest, no generation error
    eng.step(33)
    a, b, ra, rb = _both(eng, eng.ring)  # after more steps, the whole ring
    assert np.array_equal(a, b) and np.array_equal(ra, rb)
    eng.close()


def test_noalloc_digest_rejects_bad_lengths():
    """The argument checks run before any launch, with a valid output
    pointer, so that each bound is the one that fires."""
    import torch

    c = W.ten1k()
    eng = hase.Engine(64, c["seed"], c["descs"], ring_steps=40)
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    eng.step(10)
    for n, why in ((eng.ring + 1, "n_steps must be in"), (0, "n_steps must be in"), (11, "n_steps must be in")):
        with pytest.raises(hase.HaseError) as ei:
            hase.hase_digest_noalloc(eng.h, n, out.data_ptr(), None, eng.stream)
        assert ei.value.status == hase.HASE_EINVAL and why in str(ei.value), (n, str(ei.value))
    with pytest.raises(hase.HaseError) as ei:  # no output pointer
        hase.hase_digest_noalloc(eng.h, 5, 0, None, eng.stream)
    assert "out is NULL" in str(ei.value)
    hase.hase_digest_noalloc(eng.h, 10, out.data_ptr(), None, eng.stream)  # the bounds themselves are accepted
    torch.cuda.synchronize()
    eng.close()
