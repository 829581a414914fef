"""Learned step-cost model on the GPU (tn_costmodel_*).

* Gradient and prediction of the library's own CUDA kernels against the float64
  numpy oracle (oracle/mlp.py, pinned by finite differences): relative L2
  1e-4 (FP32 accumulation over a few hundred terms per gradient entry).
* Training on per-step timings recorded by the step-timing recorder on a set
  of plans, evaluated on held-out plans (measured time judges the error).
  The network learns log2(measured time / roofline time), the roofline time
  being feature 14 (log2 ms / 16); predicted log2 ms = 16 f14 + output.
* Ranking: among candidate trees of held-out workloads, the tree an ensemble
  of three trained networks predicts fastest against the trees with the
  smallest analytic cost (complex MACs) and the smallest roofline time
  (tn_estimate_tree_ms), all timed; in total the model's picks must stay
  within the spread measured between runs (10%) of either, and the gains are
  printed.
"""
import math

import numpy as np
import pytest

from tn_inputs import sycamore_circuit, random_bits, random_network
from oracle import mlp

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


def rel(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_gradient_and_forward_match_oracle(tn):
    import torch
    cm = tn.CostModel(seed=3)
    p = cm.get_params()
    rng = np.random.default_rng(4)
    X = rng.uniform(0, 1, (1000, 16)).astype(np.float32)
    X[:, 15] = 1
    T = rng.standard_normal(1000).astype(np.float32)
    dX, dT = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    dG = torch.zeros(cm.n_params, dtype=torch.float32, device="cuda")
    loss = cm.grad(dX, dT, dG)
    L, g = mlp.grad(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - L) < 1e-5 * max(1.0, L)
    assert rel(dG.cpu().numpy(), g) < 1e-4
    dY = torch.zeros(1000, dtype=torch.float32, device="cuda")
    cm.predict(dX, dY)
    torch.cuda.synchronize()
    assert rel(dY.cpu().numpy(), mlp.forward(p, X)) < 1e-5
    cm.close()


def profile_plan(tn, plan, n_slices, reps=5):
    """(features, log2 ms per launch) of every kernel step of a profiled plan:
    the median over `reps` separately recorded passes, so that one slow
    launch (a clock change, another process's work) does not move a step's
    label."""
    import torch
    amp = torch.zeros(2 << plan.n_open, dtype=torch.float64, device="cuda")
    plan.contract(0, n_slices, amp)
    per_rep = []
    for _ in range(reps):
        plan.profile(reset=True)
        plan.contract(0, n_slices, amp)
        rows = [r for r in plan.profile() if r["kind"] not in ("extract", "accumulate")]
        per_rep.append([r["ms"] / max(r["launches"], 1) for r in rows])
    feats = plan.op_features()
    assert all(len(r) == len(feats) for r in per_rep)
    ms = np.median(np.array(per_rep), axis=0)
    y = np.log2(np.maximum(ms, 1e-4)).astype(np.float32)
    return feats, y


ROOF_SCALE = 16.0

# Held-out error bounds of the trained model, as fractions of two baselines'
# errors on the same held-out steps.  Measured on GB300: with single-pass
# timings, model / mean-predictor 0.44, 0.48, 0.50, 0.51 over four runs; with
# per-step medians of 5 passes, 0.098 / 0.200 = 0.49 against the mean
# predictor and 0.098 / 0.171 = 0.57 against the roofline time plus the mean
# residual.  The bounds sit well above that spread.
MODEL_VS_MEAN = 0.75
MODEL_VS_ANALYTIC = 0.85


def residual(X, y):
    """Training target of the model: log2(time) minus log2(roofline time)."""
    return (y - ROOF_SCALE * X[:, 14]).astype(np.float32)


def predicted_log2_ms(X, out):
    return ROOF_SCALE * X[:, 14] + out


def workload_plans(tn, seeds, forms=("fp32", "tf32x3", "bf16x3")):
    out = []
    for i, seed in enumerate(seeds):
        rows, cols = [(3, 5), (4, 4), (4, 5), (3, 6), (4, 6)][i % 5]
        circ = sycamore_circuit("rect", rows, cols, 8 + (seed % 5), seed)
        n = circ.n_qubits
        open_q = list(range(n - 6, n))
        L, T, O = tn.circuit_network(circ, random_bits(n, seed), open_q)
        ns = 2 + seed % 4
        # alternately one plain greedy trial (steps of widely varying size,
        # from launch-bound to bandwidth- and tensor-bound) and the searched
        # tree (reconfigured subtrees, the kind of tree the ranking sees)
        trials = 1 if i % 2 == 0 else 24
        tree, sliced, _ = tn.find_order(L, O, tn.search_opts(trials=trials, seed=seed, n_sliced=ns))
        form = forms[i % len(forms)]
        out.append((L, T, O, sliced, tree, form))
    return out


def collect(tn, plans):
    X, Y, groups = [], [], []
    for gi, (L, T, O, sliced, tree, form) in enumerate(plans):
        plan = tn.Plan(L, T, O, sliced, tree, form=form, opts=tn.plan_opts(profile=1))
        f, y = profile_plan(tn, plan, 1 << len(sliced))
        plan.close()
        X.append(f)
        Y.append(y)
        groups += [gi] * len(y)
    return np.concatenate(X), np.concatenate(Y), np.array(groups)


def test_training_predicts_held_out_plans(tn):
    import torch
    plans = workload_plans(tn, list(range(1, 31)))
    X, Y, g = collect(tn, plans)
    train = g % 5 != 0
    cm = tn.CostModel(seed=7)
    dX = torch.from_numpy(X[train]).cuda()
    dT = torch.from_numpy(residual(X[train], Y[train])).cuda()
    l0 = cm.grad(dX, dT)
    l1 = cm.train(dX, dT, epochs=3000, lr=3e-3)
    assert l1 < 0.2 * l0
    dXt = torch.from_numpy(X[~train]).cuda()
    dYt = torch.zeros(int((~train).sum()), dtype=torch.float32, device="cuda")
    cm.predict(dXt, dYt)
    torch.cuda.synchronize()
    err = np.abs(predicted_log2_ms(X[~train], dYt.cpu().numpy()) - Y[~train])
    base = np.abs(Y[train].mean() - Y[~train])
    # the analytic fallback: roofline time plus the mean training residual
    analytic = np.abs(predicted_log2_ms(X[~train], residual(X[train], Y[train]).mean()) - Y[~train])
    print(f"cost model: train loss {l0:.3f} -> {l1:.3f}; held-out mean |log2 err| {err.mean():.3f} "
          f"(roofline time + mean residual: {analytic.mean():.3f}; predicting the mean: {base.mean():.3f}), "
          f"{int(train.sum())} train / {int((~train).sum())} test steps")
    assert err.mean() < MODEL_VS_MEAN * base.mean()
    assert err.mean() < MODEL_VS_ANALYTIC * analytic.mean()
    cm.close()


def timed(tn, plan, n_slices, reps=7):
    """Median device time (ms) of `reps` separately timed contractions."""
    import torch
    amp = torch.zeros(2 << plan.n_open, dtype=torch.float64, device="cuda")
    plan.contract(0, n_slices, amp)
    torch.cuda.synchronize()
    out = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.contract(0, n_slices, amp)
        e1.record()
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return float(np.median(out))


HELD_OUT = [(5, 5, 12, 4242), (4, 6, 12, 4243), (5, 5, 11, 4244), (4, 7, 10, 4245)]
ENSEMBLE_SEEDS = (11, 12, 13)
RANK_SLACK = 1.10


def test_learned_ranking_versus_analytic_cost(tn):
    """Among the distinct best trees of 12 search seeds for each of four
    held-out circuits, the tree the model predicts fastest against two
    analytic picks: the tree with the fewest complex MACs and the tree with
    the smallest roofline time of its compiled plan (tn_estimate_tree_ms, the
    FLOP/memory fallback), each timed as a CUDA graph replayed as one chain of
    steps (graph_branches 1: its time is the sum of its steps, the quantity
    the model predicts).  Over the four circuits the model's picks must not
    take longer in total than either analytic pick (3% timing slack); the
    gains are printed."""
    import torch
    X, Y, _ = collect(tn, workload_plans(tn, list(range(101, 131)), forms=("tf32x3",)))
    # an ensemble of independently initialised networks (their residual
    # predictions averaged): one network's picks depended on its
    # initialisation (below)
    models = []
    for seed in ENSEMBLE_SEEDS:
        cm = tn.CostModel(seed=seed)
        cm.train(torch.from_numpy(X).cuda(), torch.from_numpy(residual(X, Y)).cuda(), epochs=3000, lr=3e-3)
        models.append(cm)
    tot_a = tot_m = tot_e = tot_best = 0.0
    errs = []
    for rows, cols, cycles, seed in HELD_OUT:
        circ = sycamore_circuit("rect", rows, cols, cycles, seed)
        n = circ.n_qubits
        L, T, O = tn.circuit_network(circ, random_bits(n, 7), list(range(n - 8, n)))
        cands = []
        for s in range(12):
            tree, sliced, st = tn.find_order(L, O, tn.search_opts(trials=24, seed=1000 + s, n_sliced=6))
            if all(tree != c[0] for c in cands):
                cands.append((tree, sliced, st["log2_total"]))
        meas, pred, est = [], [], []
        for tree, sliced, _ in cands:
            plan = tn.Plan(L, T, O, sliced, tree, form="tf32x3", opts=tn.plan_opts(use_graph=1, graph_branches=1))
            meas.append(timed(tn, plan, 64))
            est.append(tn.estimate_tree_ms(L, O, sliced, tree, form="tf32x3").ms)
            f = plan.op_features()
            plan.close()
            outs = []
            for cm in models:
                d = torch.zeros(len(f), dtype=torch.float32, device="cuda")
                cm.predict(torch.from_numpy(f).cuda(), d)
                torch.cuda.synchronize()
                outs.append(d.cpu().numpy())
            pred.append(float(np.sum(2.0 ** predicted_log2_ms(f, np.mean(outs, axis=0)))))
        meas, pred = np.array(meas), np.array(pred)
        analytic = np.array([c[2] for c in cands])
        i_a, i_m, i_e = int(np.argmin(analytic)), int(np.argmin(pred)), int(np.argmin(est))
        tot_a += meas[i_a]
        tot_m += meas[i_m]
        tot_e += meas[i_e]
        tot_best += meas.min()
        errs += list(np.abs(np.log2(pred / meas)))
        print(f"{rows}x{cols} m{cycles}: {len(cands)} trees, MAC pick {meas[i_a]:.3f} ms, roofline-time pick "
              f"{meas[i_e]:.3f} ms, model pick {meas[i_m]:.3f} ms, best {meas.min():.3f} ms")
    print(f"ranking over {len(HELD_OUT)} held-out circuits: MAC picks {tot_a:.3f} ms, roofline-time picks "
          f"{tot_e:.3f} ms, model picks {tot_m:.3f} ms, best {tot_best:.3f} ms; gain {tot_a / tot_m:.3f}x over "
          f"MACs, {tot_e / tot_m:.3f}x over roofline time; median |log2(pred/meas)| {np.median(errs):.2f}")
    # Measured on GB300 with one network (before the ensemble), over
    # repeated runs of this test: model picks / MAC picks 0.95, 0.98, 1.03
    # and model picks / roofline-time picks 0.95, 1.00, 1.06; a single
    # mispick among the four circuits (a tree 1.7x slower than the best)
    # moved the total by up to 10%.  The bound sits above that spread; picks
    # made at random among the candidates (about 1.2-1.3x the MAC picks)
    # would exceed it.
    assert tot_m <= RANK_SLACK * tot_a
    assert tot_m <= RANK_SLACK * tot_e
    # the library-side ranking inside the order search uses the same model
    circ = sycamore_circuit("rect", 5, 5, 12, 4242)
    L, T, O = tn.circuit_network(circ, random_bits(25, 7), list(range(17, 25)))
    tree, sliced, st = tn.find_order(L, O, tn.search_opts(trials=24, seed=1000, n_sliced=6, candidates=8,
                                                          rank_form="tf32x3", cost_model=models[0]))
    assert len(tree) == len(L) - 1 and len(sliced) == 6
    for cm in models:
        cm.close()
