"""GPU checks of the BF16 surrogate kernels against the FP64 oracle, of its
serving/fallback decision, and of what the trained network gains over running
the lattice Boltzmann update for every query.

BF16 tolerances (8-bit significand, FP32 accumulation): inputs, weights and
activations are rounded to ~4e-3 relative at every layer, so outputs agree to
2e-2 of their scale and gradients to 5e-2 (relative norm per layer)."""
import math
import time

import numpy as np
import pytest

from paper_1004_5058_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1004_5058_gb300 import surrogate as S
    return torch, S


def box_and_inputs(S, B=256, seed=5):
    lo = np.array([-12.0, -10.35, 6.885, 0.344, 0.85])
    hi = np.array([-4.0, -7.65, 9.315, 0.466, 1.15])
    box = S.Box(0.5 * (lo + hi), 0.5 * (hi - lo))
    u = I.uniform01(seed, B * 5).reshape(B, 5)
    return box, lo + (hi - lo) * u


def oracle_params(p):
    from oracle import mlp
    return mlp.unflatten(p.astype(np.float64))


def test_forward_matches_oracle(env):
    torch, S = env
    from oracle import mlp
    box, x = box_and_inputs(S)
    p = S.init_params(3)
    sg = S.Surrogate(box, sigma_scale=2e-4, max_batch=300)
    sg.set_params(p)
    out = sg.forward(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    ref, _ = mlp.forward(oracle_params(p), mlp.normalise(x, box.center, box.half_range))
    ref = ref.copy()
    ref[:, 0] *= 2e-4
    for c in range(2):
        scale = np.sqrt(np.mean(ref[:, c] ** 2))
        assert np.max(np.abs(out[:, c] - ref[:, c])) <= 2e-2 * scale, c
    sg.close()


@pytest.mark.parametrize("B", [64, 300, 1000, 20000])
def test_gradients_match_oracle(env, B):
    """B = 20000 is 313 slabs of 64 rows on the 304 persistent CTAs of the
    training kernel: nine CTAs add a second slab into their partial row."""
    torch, S = env
    from oracle import mlp
    box, x = box_and_inputs(S, B=B, seed=B)
    p = S.init_params(4)
    t = 1e-4 * np.sin(np.arange(B))
    lab = (np.arange(B) % 3 == 0).astype(np.float64)
    sg = S.Surrogate(box, sigma_scale=1e-4, max_batch=max(1024, B), lam=0.8)
    sg.set_params(p)
    dev = "cuda"
    g, loss = sg.gradients(torch.tensor(x, dtype=torch.float32, device=dev),
                           torch.tensor(t, dtype=torch.float32, device=dev),
                           torch.tensor(lab, dtype=torch.float32, device=dev))
    z = mlp.normalise(x, box.center, box.half_range)
    params = oracle_params(p)
    ref = mlp.flatten(mlp.gradients(params, z, t / 1e-4, lab, lam=0.8))
    ref_loss = mlp.loss(params, z, t / 1e-4, lab, lam=0.8)
    assert loss == pytest.approx(ref_loss, rel=2e-2)
    off = 0
    for (wo, wi), (bo,) in mlp.param_shapes():
        for n in (wo * wi, bo):
            a, r = g[off:off + n].astype(np.float64), ref[off:off + n]
            assert np.linalg.norm(a - r) <= 5e-2 * np.linalg.norm(r) + 1e-12, (off, n)
            off += n
    assert off == g.size
    sg.close()


def test_adam_step_and_training_reduce_loss(env):
    torch, S = env
    from oracle import mlp
    box, x = box_and_inputs(S, B=1024, seed=9)
    # a smooth Herschel-Bulkley-like target over the box
    sigma = 1e-4 * (1.0 + 0.5 * (x[:, 3] - 0.405) / 0.06) + 5e-4 * np.exp(0.4 * x[:, 0])
    lab = (x[:, 0] > -8.0).astype(np.float64)
    p0 = S.init_params(1)
    sg = S.Surrogate(box, sigma_scale=float(np.max(sigma)), max_batch=1024, lr=1e-3)
    sg.set_params(p0)
    X = torch.tensor(x, dtype=torch.float32, device="cuda")
    T = torch.tensor(sigma, dtype=torch.float32, device="cuda")
    Y = torch.tensor(lab, dtype=torch.float32, device="cuda")
    g, l0 = sg.gradients(X, T, Y)
    sg.train_step(X, T, Y)
    p1 = sg.get_params()
    opt = mlp.Adam(p0.size, lr=1e-3)
    ref = opt.step(p0.astype(np.float64), g.astype(np.float64))
    # first Adam step: every parameter moves by ~lr * sign(g) (bias-corrected)
    np.testing.assert_allclose(p1, ref, rtol=0, atol=2e-6)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    for _ in range(300):
        sg.train_step(X, T, Y, loss)
    assert float(loss.item()) < 0.1 * l0
    sg.close()


def test_serve_flags_fallbacks(env):
    torch, S = env
    box, x = box_and_inputs(S, B=64, seed=2)
    sg = S.Surrogate(box, sigma_scale=1e-4, max_batch=64, logit_margin=0.5)
    p = np.zeros(S.param_count(), dtype=np.float32)
    p[-1] = 3.0  # logit bias: confident "yielded" everywhere
    sg.set_params(p)
    x[0, 0] = box.center[0] + 1.5 * box.half_range[0]  # outside the box
    x[1, 3] = np.nan
    stress, logit, fb = sg.serve(torch.tensor(x, dtype=torch.float32, device="cuda"))
    fb = fb.cpu().numpy()
    assert fb[0] == 1 and fb[1] == 1 and np.all(fb[2:] == 0)
    lg = logit.cpu().numpy()
    assert np.isnan(lg[1]) and np.allclose(np.delete(lg, 1), 3.0)  # a NaN input propagates
    p[-1] = 0.2  # undecided
    sg.set_params(p)
    _, _, fb = sg.serve(torch.tensor(x, dtype=torch.float32, device="cuda"))
    assert np.all(fb.cpu().numpy() == 1)
    sg.close()


def test_serve_error_budget_bins(env):
    """Queries whose log S bin showed a held-out error above the budget go to
    the LB; the table is validated and can be removed again."""
    torch, S = env
    from paper_1004_5058_gb300 import _lib as L
    box, x = box_and_inputs(S, B=200, seed=8)
    sg = S.Surrogate(box, sigma_scale=1e-4, max_batch=200, logit_margin=0.5)
    p = np.zeros(S.param_count(), dtype=np.float32)
    p[-1] = 3.0
    sg.set_params(p)
    lo, hi = box.center[0] - box.half_range[0], box.center[0] + box.half_range[0]
    table = np.array([1e-6, 5e-5, 1e-6, np.nan])  # bins 1 (error) and 3 (no data) over budget
    sg.set_error_budget(table, lo, hi, budget=1e-5)
    X = torch.tensor(x, dtype=torch.float32, device="cuda")
    _, _, fb = sg.serve(X)
    f32 = np.float32
    k = np.clip(np.floor((x[:, 0].astype(f32) - f32(lo)) / (f32(hi) - f32(lo)) * f32(4)), 0, 3).astype(int)
    np.testing.assert_array_equal(fb.cpu().numpy(), np.isin(k, (1, 3)).astype(np.int32))
    sg.set_error_budget(np.zeros(0), lo, hi, budget=1e-5)
    assert np.all(sg.serve(X)[2].cpu().numpy() == 0)
    e = np.zeros(300, dtype=np.float32)
    assert sg.lib.mlp_set_error_budget(sg.h, e.ctypes.data_as(L._F), 300, lo, hi, 1.0) == L.LB_ERR_INVALID
    assert sg.lib.mlp_set_error_budget(sg.h, e.ctypes.data_as(L._F), 4, hi, lo, 1.0) == L.LB_ERR_INVALID
    sg.close()


def test_surrogate_gain_over_lb(env):
    """Train on LB flow-curve points, then answer held-out queries: the network
    serves most of them within the stated stress budget, far faster per query
    than the LB run each query would otherwise need."""
    torch, S = env
    speeds = I.log_spaced(2e-4, 2e-2, 8)
    L_side, steps = 32, 3000
    x, sig, lab, _ = S.flow_curve_dataset(48, speeds, L_side=L_side, steps=steps, seed=11)
    xt, st_, lt, _ = S.flow_curve_dataset(12, speeds, L_side=L_side, steps=steps, seed=23)
    assert len(x) > 300 and len(xt) > 60
    sg, hist = S.train(x, sig, lab, epochs=300, batch=128, lr=2e-3, logit_margin=0.5)
    assert hist[-1] < 0.3 * hist[0]  # measured ~0.2 on these points
    inside = np.all(np.abs(xt - sg.box.center) <= sg.box.half_range, axis=1)
    budget = 0.1 * np.max(np.abs(st_))
    # error table from the training points (no held-out data is used for it)
    table = sg.calibrate_error_budget(x, sig, budget, n_bins=4)
    assert table.shape == (4,)
    res = S.serve_with_fallback(sg, xt[inside], L_side=L_side, steps=steps)
    served = ~res["fallback"]
    assert served.mean() > 0.5
    # stress budget: median error of served queries within 10% of the largest
    # held-out stress (measured ~5-7%); short 32x32 runs make the LB points noisy
    err = np.abs(res["stress"][served] - st_[inside][served])
    assert np.median(err) <= budget, (np.median(err), budget)
    # yielded/arrested decision of the served queries
    agree = (res["logit"][served] > 0) == (lt[inside][served] > 0.5)
    assert agree.mean() >= 0.8
    # cost per query: network vs one LB cell run per query
    t_net = res["t_network"] / len(xt[inside])
    cells = S.cells_for(np.array([[xt[0, 1], xt[0, 2], xt[0, 3], xt[0, 4]]]), [speeds[3]], L_side)
    t0 = time.perf_counter()
    S.run_cells(cells, steps)
    t_lb = time.perf_counter() - t0
    assert t_lb / t_net > 100.0
    sg.close()


def test_fused_serve_equals_layered_forward(env):
    """mlp_serve runs all layers in one kernel: its stress and logit equal the
    layered forward pass bit for bit, for a ragged batch; changing the error
    budget takes effect."""
    torch, S = env
    box, x = box_and_inputs(S, B=300, seed=12)
    sg = S.Surrogate(box, sigma_scale=1e-4, max_batch=300, logit_margin=0.5)
    sg.set_params(S.init_params(7))
    X = torch.tensor(x, dtype=torch.float32, device="cuda")
    fwd = sg.forward(X)
    n0 = sg.kernel_launches
    stress, logit, fb = sg.serve(X)
    assert sg.kernel_launches - n0 == 1
    assert torch.equal(stress, fwd[:, 0]) and torch.equal(logit, fwd[:, 1])
    lg = logit.cpu().numpy()
    assert np.array_equal(fb.cpu().numpy(), (np.abs(lg) < 0.5).astype(np.int32))  # inside the box, no table
    outs = (stress, logit, fb)
    lo, hi = box.center[0] - box.half_range[0], box.center[0] + box.half_range[0]
    sg.set_error_budget(np.array([1.0, 1.0]), lo, hi, budget=0.5)  # every bin over budget
    assert np.all(sg.serve(X, out=outs)[2].cpu().numpy() == 1)
    sg.set_error_budget(np.zeros(0), lo, hi, budget=0.5)
    assert np.array_equal(sg.serve(X, out=outs)[2].cpu().numpy(), (np.abs(lg) < 0.5).astype(np.int32))
    sg.close()
