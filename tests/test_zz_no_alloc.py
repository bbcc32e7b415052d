"""Labeling without device allocation (sw_label_from_bonds_noalloc).

For callers that may not allocate device memory (a plugin inside a host
framework that owns every device byte, or a latency-critical loop where
cudaMalloc would synchronise the device): the entry point takes device
buffers and keeps its working memory in a fixed array of the library.  Its
labels must equal those of the allocating entry point sw_label_from_bonds,
bit for bit (labels are integers), on consecutive calls that reuse the same
scratch array.  This file is collected last on purpose.
"""
from __future__ import annotations

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_7560_gb300 import build, sw
    build.build()
    return torch, sw


def test_noalloc_labels_equal_allocating_entry_point(env):
    torch, sw = env
    stream = torch.cuda.current_stream()
    # consecutive calls on the shared scratch: the largest allowed lattice,
    # then smaller ones that leave stale words of the previous call behind
    cases = [(3, 128, 0.35, 11), (2, 700, 0.5, 12), (3, 41, 0.3, 13), (2, 64, 0.9, 14)]
    assert 128 ** 3 == sw.SW_NOALLOC_MAX_SITES
    for dim, L, density, seed in cases:
        N = L ** dim
        mask = inputs.random_mask(dim, L, density, seed)
        h = sw.sw_create(sw.SW_ISING, dim, L, 2, 2.0, 1)
        try:
            ref = sw.sw_label_from_bonds(h, mask)
        finally:
            sw.sw_destroy(h)
        dmask = torch.from_numpy(mask.view(np.int32)).to("cuda")
        dlab = torch.full((N,), -7, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        sw.sw_label_from_bonds_noalloc(dim, L, dmask.data_ptr(), dlab.data_ptr(), stream.cuda_stream)
        assert np.array_equal(dlab.cpu().numpy(), ref), (dim, L)


def test_noalloc_rejects_oversized_lattice(env):
    torch, sw = env
    buf = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(sw.SwError) as e:
        sw.sw_label_from_bonds_noalloc(3, 129, buf.data_ptr(), buf.data_ptr(), 0)
    assert e.value.code == sw.SW_ERR_BAD_ARG and "too large" in str(e.value)
