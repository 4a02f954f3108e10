"""amg_pairwise_match_noalloc: the matching entry point for callers that
cannot allocate device memory (framework-owned memory pools, real-time loops
that must not allocate after start-up).  It must return exactly what
amg_pairwise_match returns, and the oracle's matching, call after call,
although its scratch array keeps the previous call's contents; and it must
not allocate: the library's allocation-failure hook stays armed while it
runs.  This file is collected last on purpose."""

import ctypes as C

import numpy as np
import pytest
import torch

from synthetic import diffusion3d, gaussian_field, poisson3d
from tests.helpers import random_spd_graph

pytestmark = pytest.mark.gpu


def _match(lib, fn, Ad):
    import paper_2406_19754_gb300 as amg

    A, keep = amg.csr_struct(*Ad)
    mate = torch.full((A.n,), 7, dtype=torch.int32, device="cuda")
    rounds = C.c_int(-1)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib, fn)(C.byref(A), C.c_void_p(mate.data_ptr()), C.byref(rounds), stream)
    torch.cuda.synchronize()
    return rc, mate.cpu().numpy(), rounds.value


def test_noalloc_matches_allocating_entry_point_twice(amg, orc):
    lib = amg._lib.load()
    cases = [poisson3d(48, 40, 36),  # 69,120 rows
             diffusion3d(np.exp(gaussian_field((30, 30, 30), 2.0, 4.0, 11))),
             random_spd_graph(500, 0.02, 4, positive_offdiag=True)]
    # values that differ across the diagonal: each edge's value from its upper row
    rp, ci, v = poisson3d(20)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    cases.append((rp, ci, np.where(ci < rows, v * (1.0 + 1e-3 * np.sin(np.arange(len(v)))), v)))
    for A in cases:
        Ad = amg.csr_to_device(A)
        rc0, want, r0 = _match(lib, "amg_pairwise_match", Ad)
        assert rc0 == 0
        # the oracle's sorted greedy matching (the same matching, Sec. 2.3)
        assert np.array_equal(want, orc.match(A))
        for _ in range(2):  # two calls in a row share the same scratch array
            # any device allocation by the library would now fail (AMG_ERR_OOM)
            lib.amg_debug_fail_alloc_after(0)
            try:
                rc, got, r = _match(lib, "amg_pairwise_match_noalloc", Ad)
            finally:
                lib.amg_debug_fail_alloc_after(-1)
            assert rc == 0
            assert np.array_equal(got, want)
            assert r == r0


def test_noalloc_rejects_rows_beyond_its_array(amg):
    lib = amg._lib.load()
    side = 65  # 274,625 rows > 262,144
    rc, _, _ = _match(lib, "amg_pairwise_match_noalloc", amg.csr_to_device(poisson3d(side)))
    assert rc == amg._lib.AMG_ERR_UNSUPPORTED
