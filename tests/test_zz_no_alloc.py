"""Allocation-free contract-all entry point (lqc_contract_all_fp64_noalloc).

Callers that cannot allocate device memory (inside a stream capture that
must not gain allocation nodes, under a host framework that owns all device
memory, in loops that must not block on an allocator) use this variant,
whose scratch is a fixed array inside the library.  Its results must match
the regular entry point (caller-provided scratch) on consecutive calls,
since every call reuses the same array.  Kept in a file of its own that
pytest collects last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_2511_02257_b300")

pytestmark = pytest.mark.gpu
TOL = 1e-12

P_i64 = ctypes.POINTER(ctypes.c_int64)
P_int = ctypes.POINTER(ctypes.c_int)


def _lib():
    lib = ctypes.CDLL(L.library_path)
    f = lib.lqc_contract_all_fp64_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, P_i64, ctypes.c_void_p, ctypes.c_int, P_i64,
                  ctypes.c_int, P_int, P_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    return f


def _arr(xs, dt, pt):
    a = np.ascontiguousarray(np.asarray(xs, dtype=dt))
    return a, a.ctypes.data_as(pt)


@pytest.mark.parametrize("lt,shape", [(1, (4, 4, 20, 20)), (64, (4, 4, 20, 20)),
                                      (700, (4, 4, 20, 20)), (4096, (4, 4, 6, 6))])
def test_noalloc_matches_regular_entry_point_twice(lt, shape):
    """lt = 4096 with one chunk per slice fills the array exactly."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    noalloc = _lib()
    sa, sb, la, ra = shape, shape, (0, 1, 2, 3), (1, 0, 3, 2)
    ea, pa = _arr(sa, np.int64, P_i64)
    eb, pb = _arr(sb, np.int64, P_i64)
    xla, pla = _arr(la, np.intc, P_int)
    xra, pra = _arr(ra, np.intc, P_int)
    nbytes = L.lqc_contract_all_scratch_bytes(lt, int(np.prod(sa)))
    scratch = torch.empty(max(nbytes, 16), dtype=torch.uint8, device="cuda")
    for call in range(2):
        rng = np.random.default_rng(100 * lt + call)
        A = rng.standard_normal((lt,) + sa) + 1j * rng.standard_normal((lt,) + sa)
        B = rng.standard_normal((lt,) + sb) + 1j * rng.standard_normal((lt,) + sb)
        dA = torch.from_numpy(A).cuda()
        dB = torch.from_numpy(B).cuda()
        ref = torch.zeros(lt, dtype=torch.complex128, device="cuda")
        got = torch.zeros(lt, dtype=torch.complex128, device="cuda")
        vp = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
        rc = L.lqc_contract_all_fp64(vp(dA), 4, pa, vp(dB), 4, pb, 4, pla, pra, lt, vp(ref),
                                     vp(scratch), None)
        assert rc == 0
        rc = noalloc(vp(dA), 4, pa, vp(dB), 4, pb, 4, pla, pra, lt, vp(got), None)
        assert rc == 0
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        # same kernels, same chunking: bit-identical; the tolerance only
        # words the failure message
        assert np.array_equal(g.view(np.float64), r.view(np.float64)), \
            np.linalg.norm(g - r) / np.linalg.norm(r)
        assert np.linalg.norm(g - r) <= TOL * np.linalg.norm(r)


@pytest.mark.parametrize("lt", [4097, 5000])
def test_noalloc_rejects_beyond_its_array(lt):
    """One slot more than the fixed array holds is rejected (the accepted
    side of the bound, lt = 4096, runs above)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    noalloc = _lib()
    ea, pa = _arr((8,), np.int64, P_i64)
    xla, pla = _arr((0,), np.intc, P_int)
    d = torch.zeros(lt * 8, dtype=torch.complex128, device="cuda")
    out = torch.zeros(lt, dtype=torch.complex128, device="cuda")
    rc = noalloc(ctypes.c_void_p(d.data_ptr()), 1, pa, ctypes.c_void_p(d.data_ptr()), 1, pa, 1,
                 pla, pla, lt, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == L.LQC_ERR_ARG
