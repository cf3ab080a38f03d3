"""GPU parity of the mixed-precision path (complex64 storage, split TF32x3 /
BF16x3 tensor-core products, FP64 correlator sums) against the oracle.

* Integer-valued operands small enough to be exact in the hi part: the
  tensor-core contraction must equal the oracle exactly (this pins the
  operand packing, the swizzled tile layout and the epilogue indexing
  independently of rounding).
* Random operands: per-contraction norm-wise relative error <= 1e-6 for
  TF32x3; whole DAGs: every correlator within 1e-6 of the FP64 oracle.
* BF16x3 error is reported, with a looser bound (16 significant bits).
"""
import ctypes

import numpy as np
import pytest

import synth
from oracle import contract as C
from oracle import dag as D

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_2511_02257_b300")

pytestmark = pytest.mark.gpu
TOL_TF32X3 = 1e-6
TOL_BF16X3 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel_err(x, ref):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


def _ext(shape):
    a = np.asarray(shape, dtype=np.int64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _pairs(xs):
    a = np.asarray(xs, dtype=np.intc)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def run_mixed(A, B, la, ra, prec):
    lt = A.shape[0]
    sa, sb = A.shape[1:], B.shape[1:]
    ea, pa = _ext(sa)
    eb, pb = _ext(sb)
    xla, pla = _pairs(la)
    xra, pra = _pairs(ra)
    nbytes = L.lqc_contract_mixed_scratch_bytes(len(sa), pa, len(sb), pb, len(la), pla, pra, lt,
                                                prec)
    assert nbytes > 0
    scratch = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    dA = torch.from_numpy(np.ascontiguousarray(A.astype(np.complex64))).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B.astype(np.complex64))).cuda()
    out_shape = (lt,) + tuple(e for i, e in enumerate(sa) if i not in la) + \
        tuple(e for j, e in enumerate(sb) if j not in ra)
    dC = torch.full(out_shape, complex("nan"), dtype=torch.complex64, device="cuda")
    rc = L.lqc_contract_mixed(_ptr(dA), len(sa), pa, _ptr(dB), len(sb), pb, len(la), pla, pra, lt,
                              prec, _ptr(dC), _ptr(scratch), None)
    assert rc == 0
    torch.cuda.synchronize()
    assert L.lqc_mixed_error(1) == 0
    return dC.cpu().numpy()


CASES = [
    ((17, 33), (33, 9), (1,), (0,)),
    ((64, 64), (64, 64), (1,), (0,)),
    ((64, 64), (64, 64), (0,), (1,)),
    ((4, 4, 19, 21), (21, 13), (3,), (0,)),
    ((4, 4, 24, 24), (4, 4, 24, 24), (1, 3), (0, 2)),
    ((12, 12, 12), (12, 12, 12), (1, 2), (0, 1)),
    ((12, 12, 12), (12, 7), (2,), (0,)),
    ((5, 3, 7, 2), (2, 7, 6), (3, 2), (0, 1)),
    ((70,), (70, 3), (0,), (0,)),
    ((3, 130), (130,), (1,), (0,)),
    ((129, 65), (65, 131), (1,), (0,)),
    ((200, 300), (300, 150), (1,), (0,)),
    ((16, 16, 16), (16, 16, 16), (1, 2), (0, 1)),   # long k: split over k
    ((40, 1100), (1100, 40), (1,), (0,)),              # k not a multiple of the tile
    # fewer rows than a tile: the exchanged product, stored transposed, with
    # the right operand K-major, or [k][n] (transposed by the converters),
    # or [k][n] with k split over partial sums
    ((13, 18), (10, 14, 18), (1,), (2,)),
    ((13, 18), (18, 10, 14), (1,), (0,)),
    ((8, 1100), (1100, 300), (1,), (0,)),
    # left operand [k][rows] read in place (a baryon over its first leg)
    ((24, 24, 24), (24, 24), (0,), (0,)),
    ((18, 130), (18, 40), (0,), (0,)),
    # left operand [outer][k][inner] read in place (a baryon over its middle
    # leg), inner extents 16, 32, 128 and 256; and exchanged into that role
    ((9, 12, 16), (12, 10), (1,), (0,)),
    ((5, 32, 32), (32, 24), (1,), (0,)),
    ((3, 16, 128), (16, 40), (1,), (0,)),
    ((2, 8, 256), (8, 20), (1,), (0,)),
    ((13, 18), (5, 18, 32), (1,), (1,)),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", [L.LQC_PREC_TF32X3, L.LQC_PREC_BF16X3])
def test_mixed_exact_on_small_integers(case, prec):
    sa, sb, la, ra = case
    lt = 3
    rng = np.random.default_rng(11)
    A = (rng.integers(-3, 4, (lt,) + sa) + 1j * rng.integers(-3, 4, (lt,) + sa))
    B = (rng.integers(-3, 4, (lt,) + sb) + 1j * rng.integers(-3, 4, (lt,) + sb))
    ref = C.contract_pair(A, B, la, ra)
    got = run_mixed(A, B, la, ra, prec)
    assert np.array_equal(got.astype(np.complex128), ref)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("lt", [1, 4])
def test_mixed_tf32x3_random(case, lt):
    sa, sb, la, ra = case
    rng = np.random.default_rng(hash((sa, sb, lt)) % 2 ** 32)
    A = (rng.standard_normal((lt,) + sa) + 1j * rng.standard_normal((lt,) + sa)).astype(np.complex64)
    B = (rng.standard_normal((lt,) + sb) + 1j * rng.standard_normal((lt,) + sb)).astype(np.complex64)
    ref = C.contract_pair(A.astype(np.complex128), B.astype(np.complex128), la, ra)
    got = run_mixed(A, B, la, ra, L.LQC_PREC_TF32X3)
    assert rel_err(got.astype(np.complex128), ref) < TOL_TF32X3
    got = run_mixed(A, B, la, ra, L.LQC_PREC_BF16X3)
    assert rel_err(got.astype(np.complex128), ref) < TOL_BF16X3


def _oracle(wl, roots=None):
    od, _ = D.build_from_workload(wl)
    cache = {}

    def lf(u):
        li = od.nodes[u].leaf_index
        if li not in cache:
            cache[li] = synth.leaf_data(wl, li)
        return cache[li]
    return od, C.evaluate(od, lf, roots)


def _run(wl, prec, roots=None, policy="tree"):
    nd, _ = L.build_dag(wl, precision=prec, leaf_data_fn=lambda li: synth.leaf_data(wl, li))
    planned = nd.schedule(policy, "lru", 0)
    nd.execute(torch.cuda.current_stream().cuda_stream)
    nd.wait()
    return nd, planned, {r: nd.read_correlator(r) for r in (roots or nd.roots())}


@pytest.mark.parametrize("seed", [0, 1])
def test_tiny_dag_tf32x3(seed):
    wl = synth.make_workload("tiny", seed=seed)
    od, ref = _oracle(wl)
    nd, planned, vals = _run(wl, "tf32x3")
    errs = [rel_err(vals[r], ref[r]) for r in ref]
    assert max(errs) < TOL_TF32X3, errs
    assert nd.stats() == planned
    # storage is complex64: half the bytes of the FP64 path
    nd64, planned64, _ = _run(wl, "fp64")
    assert planned["peak_paper"] * 2 == planned64["peak_paper"]


def test_multi_meson_tf32x3_all_roots():
    wl = synth.make_workload("multi_meson")
    od, ref = _oracle(wl)
    nd, planned, vals = _run(wl, "tf32x3")
    errs = np.array([rel_err(vals[r], ref[r]) for r in ref])
    assert errs.max() < TOL_TF32X3, (errs.max(), np.median(errs))


def test_multi_meson_bf16x3_error_reported():
    wl = synth.make_workload("multi_meson", n_functions=30)
    od, ref = _oracle(wl)
    nd, planned, vals = _run(wl, "bf16x3")
    errs = np.array([rel_err(vals[r], ref[r]) for r in ref])
    print("bf16x3 correlator error: max %.2e median %.2e" % (errs.max(), np.median(errs)))
    assert errs.max() < 1e-3


def test_baryon_tf32x3_sampled_roots():
    wl = synth.make_workload("baryon")
    od, _ = D.build_from_workload(wl)
    rng = np.random.default_rng(5)
    roots = [int(r) for r in rng.choice(od.roots(), size=24, replace=False)]
    _, ref = _oracle(wl, roots)
    nd, planned, vals = _run(wl, "tf32x3", roots)
    errs = [rel_err(vals[r], ref[r]) for r in roots]
    assert max(errs) < TOL_TF32X3, errs


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_grouped_windows_bit_identical_to_single_launches(precision):
    """Grouped window execution (independent contractions batched into a few
    launches per dependency level) performs the same arithmetic per tile as
    one launch per contraction: the correlators must agree bit for bit, with
    far fewer kernels."""
    wl = synth.make_workload("multi_meson", n_functions=40)
    nd, _ = L.build_dag(wl, precision=precision, leaf_data_fn=lambda li: synth.leaf_data(wl, li))
    nd.schedule("tree", "lru", 0)
    stream = torch.cuda.current_stream().cuda_stream
    out = {}
    kernels = {}
    for w in (0, 64, 7):
        nd.set_option(L.LQC_OPT_WINDOW, w)
        nd.execute(stream)
        out[w] = nd.read_all_correlators()
        kernels[w] = nd.exec_info()["n_kernels"]
    for w in (64, 7):
        assert np.array_equal(out[w].view(np.float64), out[0].view(np.float64)), w
    assert kernels[64] * 4 < kernels[0]
    assert kernels[64] < kernels[7] < kernels[0]     # windows hold at most W contractions


@pytest.mark.parametrize("name,kw", [
    # parts of uneven (N, Lt): a level's correlators have different slice counts
    ("batched", dict(n_dags=5, n_functions=12, nvecs=(32, 48, 64), lts=(16, 32, 64))),
    # two-baryon functions: most correlators of a level share one of 12 leaves
    ("baryon", dict(n_functions=60))])
def test_grouped_correlators_sharing_operands(name, kw):
    """A grouped level's correlators run slice by slice across its tasks, the
    tasks that share an operand next to each other (its slice is then read
    from L2 after the first).  Every block still sums the same elements in the
    same order: bit-identical to one launch per contraction, and within 1e-6
    of the oracle."""
    wl = synth.make_workload(name, seed=3, **kw)
    nd, _ = L.build_dag(wl, precision="tf32x3", leaf_data_fn=lambda li: synth.leaf_data(wl, li))
    nd.schedule("tree", "lru", 0)
    stream = torch.cuda.current_stream().cuda_stream
    out = {}
    for w in (0, 512):
        nd.set_option(L.LQC_OPT_WINDOW, w)
        nd.execute(stream)
        nd.wait()
        out[w] = nd.read_all_correlators()
    assert np.array_equal(out[512].view(np.float64), out[0].view(np.float64))
    od, _ = D.build_from_workload(wl)
    rng = np.random.default_rng(7)
    roots = [int(r) for r in rng.choice(od.roots(), size=min(16, len(od.roots())), replace=False)]
    _, ref = _oracle(wl, roots)
    errs = [rel_err(nd.read_correlator(r), ref[r]) for r in roots]
    assert max(errs) < TOL_TF32X3, errs


@pytest.mark.parametrize("case", [((16, 16), (16, 16), (0, 1), (1, 0)),
                                  ((4, 4, 20, 20), (4, 4, 20, 20), (0, 1, 2, 3), (1, 0, 3, 2)),
                                  ((4, 4, 40, 40), (4, 4, 40, 40), (0, 1, 2, 3), (1, 0, 3, 2)),
                                  ((9, 10, 11), (11, 9, 10), (0, 1, 2), (1, 2, 0)),
                                  ((33, 70), (33, 70), (0, 1), (0, 1)),
                                  ((3, 1, 50), (50, 1, 3), (0, 1, 2), (2, 1, 0)),
                                  # runs read by warps: 64, 32 (ragged), 128, 1536 = 6 x 256
                                  ((64, 64, 64), (64, 64, 64), (0, 1, 2), (1, 0, 2)),
                                  ((5, 7, 32), (7, 5, 32), (0, 1, 2), (1, 0, 2)),
                                  ((9, 10, 128), (10, 9, 128), (0, 1, 2), (1, 0, 2)),
                                  ((32, 48), (32, 48), (0, 1), (0, 1))])
@pytest.mark.parametrize("lt", [1, 5])
def test_contract_all_c64_vs_oracle(case, lt):
    """Correlator of two complex64 tensors (FP64 sums; a permuted partner is
    first reordered by the tiled transpose) against the oracle."""
    sa, sb, la, ra = case
    rng = np.random.default_rng(21)
    A = (rng.standard_normal((lt,) + sa) + 1j * rng.standard_normal((lt,) + sa)).astype(np.complex64)
    B = (rng.standard_normal((lt,) + sb) + 1j * rng.standard_normal((lt,) + sb)).astype(np.complex64)
    ref = C.contract_pair(A.astype(np.complex128), B.astype(np.complex128), la, ra)
    ea, pa = _ext(sa)
    eb, pb = _ext(sb)
    xla, pla = _pairs(la)
    xra, pra = _pairs(ra)
    nbytes = L.lqc_contract_all_c64_scratch_bytes(len(sa), pa, len(sb), pb, len(la), pla, pra, lt)
    assert nbytes > 0
    scratch = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.zeros(lt, dtype=torch.complex128, device="cuda")
    rc = L.lqc_contract_all_c64(_ptr(dA), len(sa), pa, _ptr(dB), len(sb), pb, len(la), pla, pra,
                                lt, 2.0, _ptr(dC), _ptr(scratch), None)
    assert rc == 0
    torch.cuda.synchronize()
    # products of float inputs are exact in the double-float sums: FP64-level agreement
    assert rel_err(dC.cpu().numpy(), 2.0 * ref) < 1e-12


@pytest.mark.parametrize("mkn", [(64, 64, 64), (100, 48, 130), (33, 70, 200), (256, 192, 256),
                                 (128, 1100, 96)])
@pytest.mark.parametrize("fused", [0, 1 << 30])
@pytest.mark.parametrize("window", [0, 64])
@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_matrix_product_forms_vs_oracle(mkn, fused, window, kernel):
    """C = A.B with B stored [k][n] (read in place and transposed inside the
    fused GEMM when n is even), then Tr(C.D): every form against the oracle."""
    M, K, N = mkn
    lt = 3
    rng = np.random.default_rng(M * 7 + K * 3 + N)

    def rnd(*s):
        return (rng.standard_normal((lt,) + s) + 1j * rng.standard_normal((lt,) + s)) / np.sqrt(K)
    A, B, Dm = rnd(M, K), rnd(K, N), rnd(N, M)
    ref = C.contract_pair(C.contract_pair(A, B, (1,), (0,)), Dm, (0, 1), (1, 0))
    d = L.Dag(lt, "tf32x3")
    a, b, dd = d.add_leaf((M, K), A), d.add_leaf((K, N), B), d.add_leaf((N, M), Dm)
    c = d.add_contraction(a, b, [1], [0])
    r = d.add_contraction(c, dd, [0, 1], [1, 0])
    d.schedule("tree")
    d.set_option(L.LQC_OPT_FUSED_MAX_N, fused)
    d.set_option(L.LQC_OPT_WINDOW, window)
    d.set_option(L.LQC_OPT_FUSED_KERNEL, kernel)
    d.execute(torch.cuda.current_stream().cuda_stream)
    assert rel_err(d.read_correlator(r), ref) < TOL_TF32X3
    assert L.lqc_mixed_error(1) == 0


@pytest.mark.parametrize("n", [64, 128])
@pytest.mark.parametrize("window", [0, 64])
@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_propagator_right_operand_in_place_vs_oracle(n, window, kernel):
    """M . P over P's first distillation axis: P is read in place as [k][spin
    block][n] by the fused GEMM (one 4-d TMA box per tile), then a correlator
    of the result; against the oracle."""
    lt = 2
    rng = np.random.default_rng(n + window)

    def rnd(*s):
        return (rng.standard_normal((lt,) + s) + 1j * rng.standard_normal((lt,) + s)) / np.sqrt(n)
    Mm, Pp, Dd = rnd(n, n), rnd(4, 4, n, n), rnd(n, 4, 4, n)
    ref = C.contract_pair(C.contract_pair(Mm, Pp, (1,), (2,)), Dd, (0, 1, 2, 3), (0, 1, 2, 3))
    d = L.Dag(lt, "tf32x3")
    a, b, dd = d.add_leaf((n, n), Mm), d.add_leaf((4, 4, n, n), Pp), d.add_leaf((n, 4, 4, n), Dd)
    c = d.add_contraction(a, b, [1], [2])
    r = d.add_contraction(c, dd, [0, 1, 2, 3], [0, 1, 2, 3])
    d.schedule("tree")
    d.set_option(L.LQC_OPT_FUSED_MAX_N, 1 << 30)
    d.set_option(L.LQC_OPT_WINDOW, window)
    d.set_option(L.LQC_OPT_FUSED_KERNEL, kernel)
    d.execute(torch.cuda.current_stream().cuda_stream)
    assert rel_err(d.read_correlator(r), ref) < TOL_TF32X3


@pytest.mark.parametrize("n", [32, 128])
@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_propagator_left_operand_in_place_vs_oracle(n, kernel):
    """P x P over (spin out, distillation out) and a P x M over three axes:
    left operands whose contracted axes are several groups (and whose rows are
    two groups at n = 128) are read in place; against the oracle."""
    lt = 2
    rng = np.random.default_rng(n)

    def rnd(*s):
        return (rng.standard_normal((lt,) + s) + 1j * rng.standard_normal((lt,) + s)) / np.sqrt(4 * n)
    P1, P2, Mm = rnd(4, 4, n, n), rnd(4, 4, n, n), rnd(4, 4)
    c1 = C.contract_pair(P1, P2, (1, 3), (0, 2))              # (s, i, s', j)
    ref = C.contract_pair(C.contract_pair(c1, P1, (0, 1, 3), (1, 3, 2)), Mm, (0, 1), (0, 1))
    d = L.Dag(lt, "tf32x3")
    a, b, m = d.add_leaf((4, 4, n, n), P1), d.add_leaf((4, 4, n, n), P2), d.add_leaf((4, 4), Mm)
    x = d.add_contraction(a, b, [1, 3], [0, 2])
    y = d.add_contraction(x, a, [0, 1, 3], [1, 3, 2])
    r = d.add_contraction(y, m, [0, 1], [0, 1])
    d.schedule("tree")
    d.set_option(L.LQC_OPT_FUSED_MAX_N, 1 << 30)
    d.set_option(L.LQC_OPT_FUSED_KERNEL, kernel)
    d.execute(torch.cuda.current_stream().cuda_stream)
    assert rel_err(d.read_correlator(r), ref) < TOL_TF32X3


@pytest.mark.parametrize("kernel", [0, 1, 2])
@pytest.mark.parametrize("mkn,bmn", [((40, 70, 24), True), ((130, 44, 200), True),
                                     ((129, 1100, 64), True), ((64, 48, 64), False),
                                     ((300, 34, 70), False)])
@pytest.mark.parametrize("window", [0, 64])
def test_fused_kernels_exact_on_integers(kernel, mkn, bmn, window):
    """Both fused GEMMs on small-integer operands, where the split is exact
    and every partial sum is an integer below 2^24: the correlator
    Tr(A.B.D) equals the oracle bit for bit.  Rows and k are not multiples
    of the tiles (a ragged last tile, k blocks partly beyond K), K > 512
    splits over k, and B is stored [k][n] (read in place) or [n][k]."""
    M, K, N = mkn
    lt = 3
    rng = np.random.default_rng(M + 7 * K + 13 * N + kernel)

    def ints(*s):
        return rng.integers(-3, 4, (lt,) + s) + 1j * rng.integers(-3, 4, (lt,) + s)
    A, Dm = ints(M, K), ints(N, M)
    B = ints(K, N) if bmn else ints(N, K)
    ref = C.contract_pair(C.contract_pair(A, B, (1,), (0,) if bmn else (1,)), Dm, (0, 1), (1, 0))
    d = L.Dag(lt, "tf32x3")
    a = d.add_leaf((M, K), A)
    b = d.add_leaf((K, N) if bmn else (N, K), B)
    dd = d.add_leaf((N, M), Dm)
    c = d.add_contraction(a, b, [1], [0] if bmn else [1])
    r = d.add_contraction(c, dd, [0, 1], [1, 0])
    d.schedule("tree")
    d.set_option(L.LQC_OPT_FUSED_MAX_N, 1 << 30)
    d.set_option(L.LQC_OPT_FUSED_KERNEL, kernel)
    d.set_option(L.LQC_OPT_WINDOW, window)
    d.execute(torch.cuda.current_stream().cuda_stream)
    got = d.read_correlator(r)
    assert L.lqc_mixed_error(1) == 0
    assert np.array_equal(got, ref), rel_err(got, ref)


def test_fused_kernels_agree_on_a_dag():
    """The fused GEMMs on the same DAG (multi-meson terms, every width
    fused): each within the mixed bar of the oracle on every root, and the
    CTA-pair form (kernel 2: cta_group::2 MMAs on 256-row tiles, each CTA
    converting half of the B' tile) bit-identical to the one-CTA form, whose
    per-element arithmetic it repeats."""
    wl = synth.make_workload("multi_meson", n_functions=30)
    od, _ = D.build_from_workload(wl)
    ref = C.evaluate(od, lambda u: synth.leaf_data(wl, od.nodes[u].leaf_index))
    nd, _ = L.build_dag(wl, precision="tf32x3", leaf_data_fn=lambda li: synth.leaf_data(wl, li))
    nd.schedule("tree", "lru", 0)
    nd.set_option(L.LQC_OPT_FUSED_MAX_N, 1 << 30)
    stream = torch.cuda.current_stream().cuda_stream
    worst, vals = {}, {}
    for kernel in (0, 1, 2):
        nd.set_option(L.LQC_OPT_FUSED_KERNEL, kernel)
        nd.execute(stream)
        vals[kernel] = {r: nd.read_correlator(r) for r in nd.roots()}
        assert L.lqc_mixed_error(1) == 0
        worst[kernel] = max(rel_err(vals[kernel][r], ref[r]) for r in ref)
    assert max(worst.values()) < TOL_TF32X3, worst
    for r in ref:
        assert np.array_equal(vals[2][r].view(np.float64), vals[0][r].view(np.float64)), r


@pytest.mark.parametrize("rows", [192, 256])
@pytest.mark.parametrize("window", [0, 64])
def test_pair_tiles_right_operand_in_place_vs_oracle(rows, window):
    """CTA pairs on a product of more than 128 rows whose right operand is a
    propagator read in place as [k][spin block][n] blocks (half-width boxes
    per CTA), then a correlator; against the oracle, and bit for bit against
    the one-CTA kernel."""
    n, lt = 64, 2
    rng = np.random.default_rng(rows + window)

    def rnd(*s):
        return (rng.standard_normal((lt,) + s) + 1j * rng.standard_normal((lt,) + s)) / np.sqrt(n)
    Mm, Pp, Dd = rnd(rows, n), rnd(4, 4, n, n), rnd(rows, 4, 4, n)
    ref = C.contract_pair(C.contract_pair(Mm, Pp, (1,), (2,)), Dd, (0, 1, 2, 3), (0, 1, 2, 3))
    got = {}
    for kernel in (0, 2):
        d = L.Dag(lt, "tf32x3")
        a, b, dd = d.add_leaf((rows, n), Mm), d.add_leaf((4, 4, n, n), Pp), \
            d.add_leaf((rows, 4, 4, n), Dd)
        c = d.add_contraction(a, b, [1], [2])
        r = d.add_contraction(c, dd, [0, 1, 2, 3], [0, 1, 2, 3])
        d.schedule("tree")
        d.set_option(L.LQC_OPT_FUSED_MAX_N, 1 << 30)
        d.set_option(L.LQC_OPT_WINDOW, window)
        d.set_option(L.LQC_OPT_FUSED_KERNEL, kernel)
        d.execute(torch.cuda.current_stream().cuda_stream)
        got[kernel] = d.read_correlator(r)
        assert L.lqc_mixed_error(1) == 0
    assert rel_err(got[2], ref) < TOL_TF32X3
    assert np.array_equal(got[2].view(np.float64), got[0].view(np.float64))


def test_tf32_rounding_equals_the_hardware_conversion():
    """The converters' integer TF32 rounding against cvt.rna.tf32.f32 on
    2^26 hashed float patterns (every binade, exact ties first)."""
    bad = ctypes.c_int64(-1)
    assert L.lqc_test_tf32_rounding(1 << 26, 12345, ctypes.byref(bad)) == 0
    assert bad.value == 0


def test_gemm_flops_counted_once_per_launch():
    """With per-kind timing, each GEMM launch of a level carries the flops
    of its own tasks: the counted GEMM flops equal the sum of 8 Lt M N K over
    the exterior contractions, whether a level runs one fused launch or a
    CTA-pair launch and a one-CTA launch."""
    import math
    wl = synth.make_workload("multi_meson", n_functions=30)
    nd, _ = L.build_dag(wl, precision="tf32x3", leaf_data_fn=lambda li: synth.leaf_data(wl, li))
    nd.schedule("tree", "lru", 0)
    nd.set_option(L.LQC_OPT_FUSED_MAX_N, 1 << 30)
    nd.set_option(L.LQC_OPT_TIMING, 1)
    expect = 0
    for u in range(nd.num_nodes()):
        left, right, _, _ = nd.node_operands(u)
        if left < 0 or nd.node_info(u)["rank"] == 0:
            continue
        lt = nd.node_info(u)["lt"]
        mk, kn, mn = (nd.node_info(x)["size"] // (8 * lt) for x in (left, right, u))
        k = math.isqrt(mk * kn // mn)
        expect += 8 * lt * (mk // k) * (kn // k) * k
    stream = torch.cuda.current_stream().cuda_stream
    counted = {}
    for kernel in (0, 2):
        nd.set_option(L.LQC_OPT_FUSED_KERNEL, kernel)
        nd.execute(stream)
        nd.wait()
        counted[kernel] = nd.exec_info()["flops_gemm"]
    assert counted[0] == counted[2] == expect, (counted, expect)


@pytest.mark.parametrize("kernel", [0, 2])
@pytest.mark.parametrize("window", [0, 64])
def test_left_operand_outer_k_inner_exact(kernel, window):
    """A baryon-like left operand contracted over its middle axis, [4][64][64]
    read in place as [outer][k][inner] blocks (256 rows: CTA pairs with kernel
    2), times a matrix, then a correlator: equal to the oracle bit for bit on
    small integers."""
    lt = 2
    rng = np.random.default_rng(31 + kernel + window)

    def ints(*s):
        return rng.integers(-3, 4, (lt,) + s) + 1j * rng.integers(-3, 4, (lt,) + s)
    A, Bm, Dm = ints(4, 64, 64), ints(64, 40), ints(4, 64, 40)
    ref = C.contract_pair(C.contract_pair(A, Bm, (1,), (0,)), Dm, (0, 1, 2), (0, 1, 2))
    d = L.Dag(lt, "tf32x3")
    a, b, dd = d.add_leaf((4, 64, 64), A), d.add_leaf((64, 40), Bm), d.add_leaf((4, 64, 40), Dm)
    r = d.add_contraction(d.add_contraction(a, b, [1], [0]), dd, [0, 1, 2], [0, 1, 2])
    d.schedule("tree")
    d.set_option(L.LQC_OPT_FUSED_MAX_N, 1 << 30)
    d.set_option(L.LQC_OPT_FUSED_KERNEL, kernel)
    d.set_option(L.LQC_OPT_WINDOW, window)
    d.execute(torch.cuda.current_stream().cuda_stream)
    got = d.read_correlator(r)
    assert L.lqc_mixed_error(1) == 0
    assert np.array_equal(got, ref), rel_err(got, ref)


@pytest.mark.parametrize("n", [32, 64, 128])
@pytest.mark.parametrize("kernel", [0, 2])
@pytest.mark.parametrize("window", [0, 64])
def test_left_operand_split_k_in_place_exact(n, kernel, window):
    """Propagator products whose left operand is K-major over several axes:
    P x P over (spin, distillation) has k = (spin, distillation) and rows =
    (spin, distillation) of the left operand, P x P over (spin, spin,
    distillation) has k = (merged spins, distillation) and one row axis (the
    left operand is reordered first; rows of 32, 64 and 128, CTA pairs at
    4n > 128 rows with kernel 2), then closed into correlators: equal to the
    oracle bit for bit on small integers."""
    lt = 2
    rng = np.random.default_rng(n + 7 * kernel + window)

    def ints(*s):
        return rng.integers(-2, 3, (lt,) + s) + 1j * rng.integers(-2, 3, (lt,) + s)
    P1, P2, Dx, Mm = ints(4, 4, n, n), ints(4, 4, n, n), ints(4, n, 4, n), ints(n, n)
    x = C.contract_pair(P1, P2, (1, 3), (0, 2))
    y = C.contract_pair(P1, P2, (0, 1, 3), (1, 0, 2))
    ref1 = C.contract_pair(x, Dx, (0, 1, 2, 3), (0, 1, 2, 3))
    ref2 = C.contract_pair(y, Mm, (0, 1), (0, 1))
    d = L.Dag(lt, "tf32x3")
    a, b = d.add_leaf((4, 4, n, n), P1), d.add_leaf((4, 4, n, n), P2)
    dx, m = d.add_leaf((4, n, 4, n), Dx), d.add_leaf((n, n), Mm)
    r1 = d.add_contraction(d.add_contraction(a, b, [1, 3], [0, 2]), dx, [0, 1, 2, 3],
                           [0, 1, 2, 3])
    r2 = d.add_contraction(d.add_contraction(a, b, [0, 1, 3], [1, 0, 2]), m, [0, 1], [0, 1])
    d.schedule("tree")
    d.set_option(L.LQC_OPT_FUSED_MAX_N, 1 << 30)
    d.set_option(L.LQC_OPT_FUSED_KERNEL, kernel)
    d.set_option(L.LQC_OPT_WINDOW, window)
    d.execute(torch.cuda.current_stream().cuda_stream)
    got1, got2 = d.read_correlator(r1), d.read_correlator(r2)
    assert L.lqc_mixed_error(1) == 0
    assert np.array_equal(got1, ref1), rel_err(got1, ref1)
    assert np.array_equal(got2, ref2), rel_err(got2, ref2)
