"""The allocation-free GEMM entry point (tn_gemm_split_noalloc) against the
plan-based path on the same product.

Callers that cannot allocate device memory (an allocator owned by another
framework, real-time loops) get C = A B on the tensor cores with the
library's fixed scratch array.  Calls in a row, with different shapes and
inputs, must each match the existing entry point (tn_plan_create +
tn_contract_slices on a two-tensor network, same split form) within the bound
the other tensor-core tests use for two runs of the same split arithmetic
(1e-6 relative L2; the two paths differ only in the order of split-K atomic
adds), so the shared scratch neither leaks a previous call's planes nor needs
clearing.  Against the exact product the split form's own bound applies
(1e-5: two bf16 pieces hold ~16 bits; TF32x3 is well inside it).  BF16X3 uses
2-byte planes, so its B planes sit at another offset of the scratch array than
TF32X3's; both forms run, and one case has M = 64, below the kernel's 128-row
A tile (the tile's missing rows are zero-filled by the tensor map).  A warm
call must leave the device's free memory unchanged.
This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-6        # against the plan path (same arithmetic)
TOL_EXACT = 1e-5  # against the exact complex128 product (the split's bound)


@pytest.fixture(scope="module")
def tn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2103_03074_gb300 as tn
    return tn


def rand_c64(seed, shape):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def rel(a, b):
    return float(np.linalg.norm(a.reshape(-1) - b.reshape(-1)) / np.linalg.norm(b.reshape(-1)))


def plan_product(tn, A, B, form):
    import torch
    m, k = int(np.log2(A.shape[0])), int(np.log2(A.shape[1]))
    n = int(np.log2(B.shape[1]))
    ml, kl, nl = list(range(m)), list(range(100, 100 + k)), list(range(200, 200 + n))
    plan = tn.Plan([ml + kl, kl + nl], [A.reshape((2,) * (m + k)), B.reshape((2,) * (k + n))], ml + nl, [],
                   [(0, 1)], form=form)
    amp = torch.zeros(2 * A.shape[0] * B.shape[1], dtype=torch.float64, device="cuda")
    plan.contract(0, 1, amp)
    torch.cuda.synchronize()
    plan.close()
    g = amp.cpu().numpy()
    return (g[0::2] + 1j * g[1::2]).reshape(A.shape[0], B.shape[1])


def noalloc_product(tn, A, B, form):
    import torch
    M, K = A.shape
    N = B.shape[1]
    dA = torch.from_numpy(np.ascontiguousarray(A).view(np.float32).reshape(-1)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B).view(np.float32).reshape(-1)).cuda()
    dC = torch.full((2 * M * N,), float("nan"), dtype=torch.float32, device="cuda")
    tn.gemm_split_noalloc(dA, dB, dC, M, N, K, form=form)
    torch.cuda.synchronize()
    return dC.cpu().numpy().view(np.complex64).reshape(M, N).astype(np.complex128)


@pytest.mark.parametrize("form", ["tf32x3", "bf16x3"])
def test_noalloc_matches_plan_path_two_calls(tn, form):
    # second call: smaller, different data; third: M = 64 (half an A tile)
    cases = [((512, 1024, 256), 1), ((256, 256, 64), 2), ((64, 512, 128), 3)]
    for (M, K, N), seed in cases:
        A = rand_c64(seed, (M, K))
        B = rand_c64(seed + 10, (K, N))
        ref = plan_product(tn, A, B, form)
        got = noalloc_product(tn, A, B, form)
        assert np.isfinite(got).all()
        assert rel(got, ref) < TOL
        exact = A.astype(np.complex128) @ B.astype(np.complex128)
        assert rel(got, exact) < TOL_EXACT


@pytest.mark.parametrize("form", ["tf32x3", "bf16x3"])
def test_noalloc_call_allocates_nothing(tn, form):
    import torch
    M, K, N = 256, 512, 128
    A, B = rand_c64(5, (M, K)), rand_c64(6, (K, N))
    dA = torch.from_numpy(np.ascontiguousarray(A).view(np.float32).reshape(-1)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B).view(np.float32).reshape(-1)).cuda()
    dC = torch.zeros(2 * M * N, dtype=torch.float32, device="cuda")
    tn.gemm_split_noalloc(dA, dB, dC, M, N, K, form=form)  # warm: scratch address looked up, kernels loaded
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        tn.gemm_split_noalloc(dA, dB, dC, M, N, K, form=form)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    got = dC.cpu().numpy().view(np.complex64).reshape(M, N).astype(np.complex128)
    assert rel(got, A.astype(np.complex128) @ B.astype(np.complex128)) < TOL_EXACT


def test_noalloc_rejects_oversize_and_bad_shapes(tn):
    import torch
    d = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(tn.TNError) as ei:
        tn.gemm_split_noalloc(d, d, d, 4096, 4096, 4096, form="tf32x3")  # planes far beyond 32 MiB
    assert "scratch" in str(ei.value)
    with pytest.raises(tn.TNError):
        tn.gemm_split_noalloc(d, d, d, 100, 64, 64, form="tf32x3")  # not a power of two
    with pytest.raises(tn.TNError):
        tn.gemm_split_noalloc(d, d, d, 128, 64, 64, form="fp32")  # not a split form
