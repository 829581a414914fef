"""Tensor-core split-precision GEMMs (BF16x3 and TF32x3, four real products)
on the GPU.

Single-GEMM networks exercise each operand layout (K- or M/N-contiguous), tiles
smaller than the kernel's 128 x 64 x 64 tile (zero-filled edges) and a batch
label shared by both operands.  Each result is checked twice:
  * against the exact product (complex128 numpy): relative L2 within the bound
    of the split: two bf16 pieces hold ~16 bits, so ~3 x 2^-16 per product,
    about 5e-6 in the L2 sense for random data (1e-5 asserted);
  * against a test-side emulation of the same arithmetic (round-to-nearest
    split, hi*hi + hi*lo + lo*hi, 4 real products, exact accumulation):
    agreement to 1e-6.  The kernel reads the tensor-core partial sums out into
    FP32 registers (round-to-nearest) every 512 bytes of K, so the difference
    is the tensor core's truncating accumulation over 32 MMAs plus FP32
    rounding: 6.4e-7 measured at K = 1024 (2.1e-6 when never read out, 1.5e-7
    when read out every 128 bytes).  A kernel that dropped or misplaced any
    product term would be off by ~5e-4 (tf32 lo/hi ratio) or ~4e-3 (bf16).
FP32 form: the CUDA-core kernel against the exact product, 2e-6 (FP32 sums of
up to 2048 products).  FP16S form (one fp16 piece per value after a per-operand
power-of-two scale): 2e-3 against the exact product (the bound stated for the
scaled-FP16 form; fp16 keeps 11 bits, ~3.5e-4 per GEMM), 1e-6 against its
emulation.
"""
import numpy as np
import pytest

from tn_inputs import SplitMix64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2103_03074_gb300 as tn
    return tn


def bf16(x):
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def tf32(x):
    # round to nearest, ties away from zero, on a 10-bit mantissa
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return r.view(np.float32)


def emulate_split_4m(a, b, rnd):
    def parts(x):
        h = rnd(x)
        return h.astype(np.float64), rnd(np.asarray(x, np.float32) - h).astype(np.float64)

    def rmm(x, y):
        xh, xl = parts(x)
        yh, yl = parts(y)
        return xh @ yh + xh @ yl + xl @ yh
    ar, ai = a.real.astype(np.float32), a.imag.astype(np.float32)
    br, bi = b.real.astype(np.float32), b.imag.astype(np.float32)
    return (rmm(ar, br) - rmm(ai, bi)) + 1j * (rmm(ar, bi) + rmm(ai, br))


def emulate_fp16s_4m(a, b):
    """Scaled FP16 form: each operand scaled by 2^-e (e from its max |re|,|im|
    so the largest scaled value lies in [2^13, 2^14)), rounded to fp16, four
    real products accumulated exactly, result scaled back by 2^(eA + eB)."""
    def scaled(x):
        mx = max(np.abs(x.real).max(), np.abs(x.imag).max())
        e = np.frexp(np.float32(mx))[1] - 14
        xs = (x.astype(np.complex64) * np.float32(2.0 ** -e))
        return (xs.real.astype(np.float16).astype(np.float64), xs.imag.astype(np.float16).astype(np.float64), e)
    ar, ai, ea = scaled(a)
    br, bi, eb = scaled(b)
    return ((ar @ br - ai @ bi) + 1j * (ar @ bi + ai @ br)) * 2.0 ** (ea + eb)


def emulate_fp16x3_4m(a, b):
    """Scaled FP16 hi/lo form: each operand scaled by 2^-e as in the FP16S
    form, hi = fp16(x), lo = fp16(x - hi) (round to nearest, subnormals
    kept), hi*hi + hi*lo + lo*hi per real product, four real products
    accumulated exactly, result scaled back by 2^(eA + eB)."""
    def scaled(x):
        mx = max(np.abs(x.real).max(), np.abs(x.imag).max())
        e = np.frexp(np.float32(mx))[1] - 14
        xs = x.astype(np.complex64) * np.float32(2.0 ** -e)

        def parts(v):
            v = np.asarray(v, np.float32)
            h = v.astype(np.float16)
            lo = (v - h.astype(np.float32)).astype(np.float16)
            return h.astype(np.float64), lo.astype(np.float64)
        return parts(xs.real), parts(xs.imag), e

    def rmm(x, y):
        return x[0] @ y[0] + x[0] @ y[1] + x[1] @ y[0]
    ar, ai, ea = scaled(a)
    br, bi, eb = scaled(b)
    return ((rmm(ar, br) - rmm(ai, bi)) + 1j * (rmm(ar, bi) + rmm(ai, br))) * 2.0 ** (ea + eb)


def emulate_split_3m(a, b, form):
    """Gauss's 3M product of the split forms: T1 = A_re B_re, T2 = A_im B_im,
    T3 = (A_re + A_im)(B_re + B_im) with the sums rounded to FP32 (after the
    power-of-two scale for FP16X3), each real product hi*hi + hi*lo + lo*hi
    of round-to-nearest pieces accumulated exactly; re = T1 - T2,
    im = T3 - T1 - T2."""
    def scale_of(x):
        if form != "fp16x3":
            return 0
        mx = max(np.abs(x.real).max(), np.abs(x.imag).max())
        return int(np.frexp(np.float32(mx))[1] - 14)

    def parts(v):
        v = np.asarray(v, np.float32)
        if form == "fp16x3":
            h = v.astype(np.float16).astype(np.float32)
            lo = (v - h).astype(np.float16).astype(np.float32)
        else:
            rnd = bf16 if form == "bf16x3" else tf32
            h = rnd(v)
            lo = rnd(v - h)
        return h.astype(np.float64), lo.astype(np.float64)

    def rmm(x, y):
        xh, xl = parts(x)
        yh, yl = parts(y)
        return xh @ yh + xh @ yl + xl @ yh
    ea, eb = scale_of(a), scale_of(b)
    a = a.astype(np.complex64) * np.float32(2.0 ** -ea)
    b = b.astype(np.complex64) * np.float32(2.0 ** -eb)
    ar, ai = a.real.astype(np.float32), a.imag.astype(np.float32)
    br, bi = b.real.astype(np.float32), b.imag.astype(np.float32)
    t1, t2, t3 = rmm(ar, br), rmm(ai, bi), rmm(ar + ai, br + bi)
    return ((t1 - t2) + 1j * (t3 - t1 - t2)) * 2.0 ** (ea + eb)


def rand_c64(seed, shape):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def rel(a, b):
    return float(np.linalg.norm(a.reshape(-1) - b.reshape(-1)) / np.linalg.norm(b.reshape(-1)))


@pytest.mark.parametrize("m,k,n,a_kfirst,b_nfirst", [
    (10, 10, 8, False, False),   # A [m][k] (K contiguous), B [k][n] (N contiguous)
    (10, 9, 8, True, True),      # A [k][m] (M contiguous), B [n][k] (K contiguous)
    (6, 7, 6, False, True),      # M = 64 < 128-row tile: zero-filled rows
    (8, 5, 8, True, True),       # K = 32 < 64-wide chunk: zero-filled K
    (9, 4, 9, False, True),      # K = 16: zero-filled K in the tile
    (10, 9, 4, True, True),      # N = 16: zero-filled B rows in the tile
    (10, 3, 10, True, False),    # K = 8 (a 16-byte bf16 plane row)
    (9, 11, 6, True, False),
])
def test_single_gemm_bf16x3(tn, m, k, n, a_kfirst, b_nfirst):
    import torch
    M, K, N = 1 << m, 1 << k, 1 << n
    A = rand_c64(m * 100 + k, (M, K))
    B = rand_c64(n * 100 + k + 1, (K, N))
    ml = list(range(0, m))
    kl = list(range(100, 100 + k))
    nl = list(range(200, 200 + n))
    la = (kl + ml) if a_kfirst else (ml + kl)
    ta = (A.T if a_kfirst else A).reshape((2,) * (m + k))
    lb = (nl + kl) if b_nfirst else (kl + nl)
    tb = (B.T if b_nfirst else B).reshape((2,) * (k + n))
    open_l = ml + nl
    exact = A.astype(np.complex128) @ B.astype(np.complex128)
    emu = {"bf16x3": emulate_split_4m(A, B, bf16), "tf32x3": emulate_split_4m(A, B, tf32),
           "fp16s": emulate_fp16s_4m(A, B), "fp16x3": emulate_fp16x3_4m(A, B)}
    for form, tol_exact in (("fp32", 2e-6), ("bf16x3", 1e-5), ("tf32x3", 1e-6), ("fp16x3", 1e-6),
                            ("fp16s", 2e-3)):
        plan = tn.Plan([la, lb], [ta, tb], open_l, [], [(0, 1)], form=form)
        amp = torch.zeros(2 * M * N, dtype=torch.float64, device="cuda")
        plan.contract(0, 1, amp)
        torch.cuda.synchronize()
        g = amp.cpu().numpy()
        got = (g[0::2] + 1j * g[1::2]).reshape(M, N)
        assert rel(got, exact) < tol_exact, form
        if form != "fp32":
            assert rel(got, emu[form]) < 1e-6, form
        if form == "bf16x3":
            assert rel(emu[form], exact) > 1e-6  # the split form really is coarser than FP32
        plan.close()


@pytest.mark.parametrize("form", ["bf16x3", "tf32x3", "fp16x3", "fp16s"])
def test_batched_gemm_split(tn, form):
    """A sliced label shared by both operands becomes a batch label of the
    GEMM when the slices run as one batch."""
    import torch
    m, k, n = 8, 7, 7
    M, K, N = 1 << m, 1 << k, 1 << n
    ml, kl, nl = list(range(m)), list(range(100, 100 + k)), list(range(200, 200 + n))
    h = 300  # two batch labels
    la = [h, h + 1] + ml + kl
    lb = [h, h + 1] + kl + nl
    A = rand_c64(5, (4, M, K))
    B = rand_c64(6, (4, K, N))
    plan = tn.Plan([la, lb], [A.reshape((2,) * (m + k + 2)), B.reshape((2,) * (k + n + 2))], ml + nl,
                   [h, h + 1], [(0, 1)], form=form, opts=tn.plan_opts(batch_log2=2))
    amp = torch.zeros(2 * M * N, dtype=torch.float64, device="cuda")
    plan.contract(0, 4, amp)
    torch.cuda.synchronize()
    g = amp.cpu().numpy()
    got = (g[0::2] + 1j * g[1::2]).reshape(M, N)
    # slice s: label h takes bit 0 of s, label h+1 bit 1; A index (h, h+1) -> 2*b0 + b1
    exact = sum(A[2 * (s & 1) + (s >> 1)].astype(np.complex128) @ B[2 * (s & 1) + (s >> 1)].astype(np.complex128)
                for s in range(4))
    assert rel(got, exact) < (2e-3 if form == "fp16s" else 1e-5)
    plan.close()


# 3M against its emulation: the tensor core's truncating accumulation over the
# MMAs between read-outs, as for the 4M form (<= 1e-6 there), on sums that are
# about twice as large (T3 holds (A_re + A_im)(B_re + B_im)) and partly
# cancel in im = T3 - T1 - T2: 3e-6 allowed.  A dropped or misplaced product
# term is off by ~5e-4 (tf32) or ~4e-3 (bf16).
TOL_3M_EMU = 3e-6


@pytest.mark.parametrize("m,k,n,a_kfirst,b_nfirst", [
    (10, 10, 8, False, False),
    (10, 9, 8, True, True),
    (6, 7, 6, False, True),      # M = 64 < 128-row tile
    (9, 4, 9, False, True),      # K = 16
    (10, 3, 10, True, False),    # K = 8: a 16-byte fp16 plane row inside the 32-byte chunk
    (9, 11, 6, True, False),
])
@pytest.mark.parametrize("form", ["tf32x3", "fp16x3", "bf16x3"])
def test_single_gemm_3m(tn, form, m, k, n, a_kfirst, b_nfirst):
    """The 3M product (tc_products 3, six planes per operand, 9 MMAs of
    128 x 64 per K step) against the exact product at the form's bound and
    against the emulation of the same split arithmetic."""
    import torch
    M, K, N = 1 << m, 1 << k, 1 << n
    A = rand_c64(m * 100 + k + 7, (M, K))
    B = rand_c64(n * 100 + k + 8, (K, N))
    ml, kl, nl = list(range(0, m)), list(range(100, 100 + k)), list(range(200, 200 + n))
    la = (kl + ml) if a_kfirst else (ml + kl)
    ta = (A.T if a_kfirst else A).reshape((2,) * (m + k))
    lb = (nl + kl) if b_nfirst else (kl + nl)
    tb = (B.T if b_nfirst else B).reshape((2,) * (k + n))
    plan = tn.Plan([la, lb], [ta, tb], ml + nl, [], [(0, 1)], form=form, opts=tn.plan_opts(tc_products=3))
    assert "tensor-core 3M" in plan.describe()
    amp = torch.zeros(2 * M * N, dtype=torch.float64, device="cuda")
    plan.contract(0, 1, amp)
    torch.cuda.synchronize()
    plan.close()
    g = amp.cpu().numpy()
    got = (g[0::2] + 1j * g[1::2]).reshape(M, N)
    exact = A.astype(np.complex128) @ B.astype(np.complex128)
    emu = emulate_split_3m(A, B, form)
    print(f"3M {form} {M}x{K}x{N}: vs exact {rel(got, exact):.2e}, vs emulation {rel(got, emu):.2e}")
    assert rel(got, exact) < (3e-5 if form == "bf16x3" else 1e-6 * 3)
    assert rel(got, emu) < TOL_3M_EMU


@pytest.mark.parametrize("form", ["tf32x3", "fp16x3"])
def test_batched_gemm_3m_matches_4m(tn, form):
    """A batched GEMM (two batch labels) in the 3M and the 4M product: both
    within the form's bound of the exact sum, and of each other."""
    import torch
    m, k, n = 9, 8, 7
    M, K, N = 1 << m, 1 << k, 1 << n
    ml, kl, nl = list(range(m)), list(range(100, 100 + k)), list(range(200, 200 + n))
    h = 300
    A = rand_c64(15, (4, M, K))
    B = rand_c64(16, (4, K, N))
    exact = sum(A[2 * (s & 1) + (s >> 1)].astype(np.complex128) @ B[2 * (s & 1) + (s >> 1)].astype(np.complex128)
                for s in range(4))
    got = {}
    for prod in (3, 4):
        plan = tn.Plan([[h, h + 1] + ml + kl, [h, h + 1] + kl + nl],
                       [A.reshape((2,) * (m + k + 2)), B.reshape((2,) * (k + n + 2))], ml + nl, [h, h + 1],
                       [(0, 1)], form=form, opts=tn.plan_opts(batch_log2=2, tc_products=prod))
        amp = torch.zeros(2 * M * N, dtype=torch.float64, device="cuda")
        plan.contract(0, 4, amp)
        torch.cuda.synchronize()
        plan.close()
        g = amp.cpu().numpy()
        got[prod] = (g[0::2] + 1j * g[1::2]).reshape(M, N)
        assert rel(got[prod], exact) < 3e-6
    assert rel(got[3], got[4]) < 5e-6


@pytest.mark.parametrize("form", ["tf32x3", "fp16x3", "bf16x3"])
def test_single_gemm_3m_64_byte_chunks(tn, form):
    """The 3M kernel with 64-byte K chunks (two ring stages, two MMA K steps
    per stage, tc_chunk_bytes 64) against the same emulation and bound."""
    import torch
    M, K, N = 1024, 1024, 256
    A = rand_c64(71, (M, K))
    B = rand_c64(72, (K, N))
    ml, kl, nl = list(range(0, 10)), list(range(100, 110)), list(range(200, 208))
    plan = tn.Plan([ml + kl, kl + nl], [A.reshape((2,) * 20), B.reshape((2,) * 18)], ml + nl, [], [(0, 1)],
                   form=form, opts=tn.plan_opts(tc_products=3, tc_chunk_bytes=64))
    amp = torch.zeros(2 * M * N, dtype=torch.float64, device="cuda")
    plan.contract(0, 1, amp)
    torch.cuda.synchronize()
    plan.close()
    g = amp.cpu().numpy()
    got = (g[0::2] + 1j * g[1::2]).reshape(M, N)
    exact = A.astype(np.complex128) @ B.astype(np.complex128)
    assert rel(got, exact) < (3e-5 if form == "bf16x3" else 3e-6)
    assert rel(got, emulate_split_3m(A, B, form)) < TOL_3M_EMU


@pytest.mark.parametrize("form", ["fp16x3", "bf16x3", "fp16s"])
def test_planar_tma_store(tn, form):
    """A GEMM whose output is the next GEMM's 16-bit planes, with several
    accumulator read-outs per tile (K = 2^9), writes the planes to shared
    memory in the order of a destination box and stores them by TMA ("tma
    box=" in its plan line).  The two-GEMM product (A B) D against the same
    plan with the planes stored by the epilogue warps (tc_tma_store -1) --
    the same pieces in the same places, so the results are identical -- and
    against a separate split pass (tc_planar -1) and the exact product, with
    the bounds of the planar-epilogue parity test."""
    import torch
    m, k, n, p = 14, 9, 9, 4
    ml, kl, nl, pl = (list(range(b, b + c)) for b, c in ((0, m), (100, k), (200, n), (400, p)))
    A = rand_c64(91, (1 << m, 1 << k))
    B = rand_c64(92, (1 << k, 1 << n))
    D = rand_c64(93, (1 << n, 1 << p))
    labels = [ml + kl, kl + nl, nl + pl]
    tensors = [A.reshape((2,) * (m + k)), B.reshape((2,) * (k + n)), D.reshape((2,) * (n + p))]
    got = {}
    for key, opts in (("tma", dict()), ("staged", dict(tc_tma_store=-1)), ("split", dict(tc_planar=-1))):
        plan = tn.Plan(labels, tensors, ml + pl, [], [(0, 1), (3, 2)], form=form, opts=tn.plan_opts(**opts))
        first = [l for l in plan.describe().splitlines() if "gemm" in l][0]
        assert ("tma box=" in first) == (key == "tma"), first
        amp = torch.zeros(2 << (m + p), dtype=torch.float64, device="cuda")
        plan.contract(0, 1, amp)
        torch.cuda.synchronize()
        plan.close()
        g = amp.cpu().numpy()
        got[key] = g[0::2] + 1j * g[1::2]
    exact = ((A.astype(np.complex128) @ B.astype(np.complex128)) @ D.astype(np.complex128)).reshape(-1)
    agree = {"fp16x3": 5e-6, "fp16s": 2e-3}.get(form, 1e-6)
    bound = {"bf16x3": 1e-4, "fp16s": 2e-3}.get(form, 1e-5)
    print(f"{form}: tma vs staged {rel(got['tma'], got['staged']):.2e}, vs split pass "
          f"{rel(got['tma'], got['split']):.2e}, vs exact {rel(got['tma'], exact):.2e}")
    assert rel(got["tma"], got["staged"]) < 1e-7
    assert rel(got["tma"], got["split"]) < agree
    assert rel(got["tma"], exact) < bound
