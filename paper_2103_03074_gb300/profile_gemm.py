"""Run one pairwise contraction of a chosen GEMM shape through the C ABI, for
profiling a single kernel in isolation (e.g. under ncu):

    python -m paper_2103_03074_gb300.profile_gemm --h 2 --m 13 --k 11 --n 9 --form tf32x3 --reps 3

Shapes are log2 sizes: two tensors A[h, m, k] and B[h, k, n] with random
complex64 entries; the h labels are sliced and kept as batch labels, so the
step is a batched GEMM.  Prints the mean device time per contraction.
"""
import argparse
import sys

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--h", type=int, default=0)
    ap.add_argument("--m", type=int, default=13)
    ap.add_argument("--k", type=int, default=11)
    ap.add_argument("--n", type=int, default=9)
    ap.add_argument("--form", default="tf32x3")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--chunk", type=int, default=0, help="tensor-core K chunk bytes (64/128, 0 = default)")
    ap.add_argument("--flush", type=int, default=0, help="K bytes between accumulator read-outs (0 = default)")
    a = ap.parse_args()
    import torch
    import paper_2103_03074_gb300 as tn
    rng = np.random.default_rng(0)
    hl = list(range(300, 300 + a.h))
    ml, kl, nl = list(range(a.m)), list(range(100, 100 + a.k)), list(range(200, 200 + a.n))
    ra, rb = a.h + a.m + a.k, a.h + a.k + a.n
    A = (rng.standard_normal(1 << ra) + 1j * rng.standard_normal(1 << ra)).astype(np.complex64)
    B = (rng.standard_normal(1 << rb) + 1j * rng.standard_normal(1 << rb)).astype(np.complex64)
    plan = tn.Plan([hl + ml + kl, hl + kl + nl], [A.reshape((2,) * ra), B.reshape((2,) * rb)], ml + nl, hl,
                   [(0, 1)], form=a.form, opts=tn.plan_opts(batch_log2=a.h, tc_chunk_bytes=a.chunk,
                                                   tc_flush_bytes=a.flush))
    amp = torch.zeros(2 << (a.m + a.n), dtype=torch.float64, device="cuda")
    plan.contract(0, 1 << a.h, amp)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        plan.contract(0, 1 << a.h, amp)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    macs = float(1 << (a.h + a.m + a.k + a.n))
    print(f"h={a.h} m={a.m} k={a.k} n={a.n} form={a.form} chunk={a.chunk} flush={a.flush}: {ms:.3f} ms per contraction, "
          f"{8 * macs / ms / 1e9:.1f} complex TFLOP/s (all kernels of the step)")
    plan.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
