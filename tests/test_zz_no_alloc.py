"""The allocation-free Newton sign entry point (lq_newton_sign_noalloc).

Some callers cannot let this library allocate device memory -- a process whose GPU memory
belongs entirely to a pool allocator, or a service that allows no allocation after start-up.
For them the batched Newton sign has a variant whose workspace is a static device array.  This
test calls it through the C ABI and checks it against the allocating entry point
(lq_newton_sign) on two calls in a row, so that contents left in the shared array by the
first call cannot leak into the second.  It lives in its own file, collected last."""
import ctypes

import numpy as np
import pytest
import torch

from tests.helpers import relerr

pytestmark = pytest.mark.gpu


def _batch(rng, nb, k):
    lam = (0.5 + np.abs(rng.standard_normal((nb, k)))) * np.where(rng.random((nb, k)) < 0.5, -1, 1) \
        + 0.2j * rng.standard_normal((nb, k))
    Q = rng.standard_normal((nb, k, k)) + 1j * rng.standard_normal((nb, k, k)) + 3 * np.eye(k)
    return np.einsum("bij,bj,bjk->bik", Q, lam, np.linalg.inv(Q))


def test_noalloc_matches_allocating_entry_point(lqlib):
    from paper_1611_00195_gb300 import lq
    rng = np.random.default_rng(2024)
    ctx = lq.Context((2, 2, 2, 2))
    ctx.reserve(128, 8, False)
    for nb, k in [(8, 128), (3, 37)]:          # two calls in a row, the second smaller
        X = torch.from_numpy(_batch(rng, nb, k)).cuda()
        S0, it0 = ctx.newton_sign(X)
        S1, it1 = lq.newton_sign_noalloc(X)
        S0, S1 = S0.cpu().numpy(), S1.cpu().numpy()
        assert it1 == it0
        for b in range(nb):
            assert relerr(S1[b], S0[b]) < 1e-11
            assert np.abs(S1[b] @ S1[b] - np.eye(k)).max() < 1e-9


def test_noalloc_rejects_sizes_beyond_its_workspace(lqlib):
    from paper_1611_00195_gb300 import lq
    L = lq.lib()
    X = torch.zeros((1, 129, 129), dtype=torch.complex128, device="cuda")
    S = torch.zeros_like(X)
    it = (ctypes.c_int * 1)()
    code = L.lq_newton_sign_noalloc(ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(S.data_ptr()), 129, 1, 50, 1e-13,
                                    it, None)
    assert code == -1
    X9 = torch.zeros((9, 4, 4), dtype=torch.complex128, device="cuda")
    code = L.lq_newton_sign_noalloc(ctypes.c_void_p(X9.data_ptr()), ctypes.c_void_p(X9.data_ptr()), 4, 9, 50, 1e-13,
                                    it, None)
    assert code == -1


def test_noalloc_rejects_host_pointers(lqlib):
    # a host buffer in either argument comes back as LQ_ERR_LAYOUT before any kernel runs;
    # the device context stays usable afterwards
    from paper_1611_00195_gb300 import lq
    L = lq.lib()
    k = 4
    Xh = np.eye(k, dtype=np.complex128)[None].copy()
    Sh = np.zeros_like(Xh)
    Xd = torch.from_numpy(Xh).cuda()
    Sd = torch.zeros_like(Xd)
    it = (ctypes.c_int * 1)()
    for xp, sp in [(Xh.ctypes.data, Sd.data_ptr()), (Xd.data_ptr(), Sh.ctypes.data), (Xh.ctypes.data, Sh.ctypes.data)]:
        code = L.lq_newton_sign_noalloc(ctypes.c_void_p(xp), ctypes.c_void_p(sp), k, 1, 50, 1e-13, it, None)
        assert code == lq.LQ_ERR_LAYOUT
    with pytest.raises(TypeError):
        lq.newton_sign_noalloc(Xh)
    torch.cuda.synchronize()
    S, _ = lq.newton_sign_noalloc(Xd)
    assert np.abs(S.cpu().numpy()[0] - np.eye(k)).max() < 1e-14
