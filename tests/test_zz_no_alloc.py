"""The no-allocation query projection (pmlsh_project_noalloc).

It serves callers that cannot let a library call cudaMalloc (a process whose
device memory is owned by its own allocator, or a latency-critical loop that
must not take cudaMalloc's device-wide synchronisation).  Its output must
equal pmlsh_project's, through the C ABI, on consecutive calls that reuse the
library's static staging array.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_05537_gb300 as pm  # noqa: E402


def _noalloc(ix, Q, o64, o32):
    return pm.lib().pmlsh_project_noalloc(
        ix._h, ctypes.c_void_p(Q.data_ptr()), Q.shape[0], ctypes.c_void_p(o64.data_ptr()),
        ctypes.c_void_p(o32.data_ptr()), pm._stream())


def test_project_noalloc_matches_project():
    # d = 100 pads each row to 128 columns in the staging array
    X, Q, _, _ = datagen.mixture(3000, 100, 10, 1.0, seed=5, nq=700)
    A = oracle.gen_projection(3, 15, 100).astype(np.float32)
    ix = pm.Index(torch.from_numpy(X).cuda(), proj=A, leaf_size=64)
    Qd = torch.from_numpy(Q).cuda()
    ref64, ref32 = ix.project(Qd)
    torch.cuda.synchronize()
    ref64, ref32 = ref64.cpu().numpy(), ref32.cpu().numpy()
    # two calls in a row: the second finds the first call's rows in the array
    for rows in (Qd, Qd[:333].contiguous()):
        o64 = torch.full((rows.shape[0], 15), float("nan"), dtype=torch.float64, device="cuda")
        o32 = torch.full((rows.shape[0], 15), float("nan"), dtype=torch.float32, device="cuda")
        assert _noalloc(ix, rows, o64, o32) == 0, pm.lib().pmlsh_last_error()
        torch.cuda.synchronize()
        n = rows.shape[0]
        # same tolerance as the projection parity tests: bit-identical values
        assert np.array_equal(o64.cpu().numpy(), ref64[:n])
        assert np.array_equal(o32.cpu().numpy(), ref32[:n])
    # batches beyond the stated limit are refused, nothing is written
    big = torch.zeros((4_194_304 // 128 + 1, 100), dtype=torch.float32, device="cuda")
    o64 = torch.zeros((big.shape[0], 15), dtype=torch.float64, device="cuda")
    o32 = torch.zeros((big.shape[0], 15), dtype=torch.float32, device="cuda")
    assert _noalloc(ix, big, o64, o32) == 1
    assert b"no-allocation limit" in pm.lib().pmlsh_last_error()
    ix.close()
