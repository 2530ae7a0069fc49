"""The allocation-free entry point tg_morton_sort_noalloc, called through the C ABI.

It serves callers that cannot allocate device memory (memory owned by another allocator or held
to a fixed budget, or loops that must not take an allocation's device synchronisation).  Its
output must equal what the allocating path computes (tg_build_tree): the sort is integer work,
so the comparison is bit for bit.  Two calls in a row check that the shared static scratch holds
no state that leaks from one call into the next.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_1712_10116_gb300 import ics

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1712_10116_gb300 import binding as tg


def _reference(pos):
    s = tg.Solver(tg.Params(p=3, n_crit=64))
    tg.tg_build_tree(s.ctx, pos)
    t = tg.tg_get_tree(s.ctx)
    s.close()
    return t["keys"], t["perm"]


def test_noalloc_sort_matches_allocating_path_twice():
    dev = torch.device("cuda:0")
    # 98 and 38 sort tiles, the largest size the static scratch is laid out for (128 full tiles),
    # and a size just below it that ends in a ragged tile
    nmax = tg.TG_NOALLOC_MAX_N
    cases = [ics.plummer(200003, 1001)[0], ics.clustered(77777, 1007)[0], ics.uniform_sphere(nmax, 1002)[0],
             ics.plummer(nmax - 2047 - 64, 1008)[0]]
    for pos_np in cases:
        pos = torch.tensor(np.ascontiguousarray(pos_np), device=dev)
        keys, perm = tg.tg_morton_sort_noalloc(pos)
        torch.cuda.synchronize()
        want_keys, want_perm = _reference(pos)
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), want_keys)
        assert np.array_equal(perm.cpu().numpy(), want_perm)


def test_noalloc_rejects_sizes_beyond_its_limit():
    dev = torch.device("cuda:0")
    n = tg.TG_NOALLOC_MAX_N + 1
    pos = torch.zeros((3, n), dtype=torch.float64, device=dev)
    with pytest.raises(tg.TGError):
        tg.tg_morton_sort_noalloc(pos)
