"""GPU parity of the learned warm start: the hand-written BF16/FP32 network
kernels against the oracle's FP64 network evaluated with the same bf16
storage points, the problem-side features / targets / energy-scaled start
against their oracle definitions, and the fallback to plain PCG."""
import json

import numpy as np
import pytest

import workloads as W
from oracle import fem, nn, warm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def topo():
    import __graft_entry__ as g
    g.build()
    from paper_2012_08208_gb300 import topo as t
    return t


def _bf16_tensor(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to("cuda").to(torch.bfloat16)


def _params(widths, c_in, seed):
    """He-initialised weights rounded to bf16, small nonzero FP32 biases."""
    rng = np.random.default_rng(seed + 100)
    out = []
    for w, b in nn.init_params(seed=seed, c_in=c_in, c_out=3, widths=widths):
        out.append((nn.to_bf16(w), rng.normal(0.0, 0.05, size=b.shape).astype(np.float32).astype(np.float64)))
    return out


CASES = [((16, 32, 64, 64), 8, 2, (8, 16, 24)), ((16, 16, 32, 32), 5, 1, (16, 8, 8))]


def _int_params(widths, c_in, seed, k=3.0):
    """Sparse weights in {-1, 0, 1} (about k nonzero taps per output) and biases
    in {0, 1}: with integer inputs every activation is a short dyadic number,
    so FP32 and FP64 sums are exact and both sides round to bf16 identically."""
    rng = np.random.default_rng(seed)
    out = []
    for co, ci in nn.layer_shapes(c_in, 3, widths):
        q = k / (27 * ci)
        out.append((rng.choice([-1.0, 0.0, 1.0], size=(co, ci, 27), p=[q / 2, 1 - q, q / 2]),
                    rng.integers(0, 2, size=co).astype(np.float64)))
    return out


def _run(topo, params, widths, c_in, x, gy):
    n, _, D, H, Wd = x.shape
    net = topo.Net(c_in, widths)
    net.set_params(params)
    xt = _bf16_tensor(x)
    y = torch.empty((n, 3, D, H, Wd), dtype=torch.float32, device="cuda")
    net.zero_grad()
    net.forward(xt, y)
    net.backward(torch.from_numpy(gy.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    out = y.cpu().numpy(), topo.unpack_params(net.get_grads(), net.shapes)
    net.close()
    return out


def _oracle(params, x, gy):
    ys, tot = [], None
    for s in range(x.shape[0]):
        y, cache = nn.forward(params, x[s], keep=True, quant=nn.to_bf16)
        g = nn.backward(params, cache, gy[s].astype(np.float64))
        ys.append(y)
        tot = g if tot is None else [(a + c, b + d) for (a, b), (c, d) in zip(tot, g)]
    return np.stack(ys), tot


@pytest.mark.parametrize("widths,c_in,n,shape", CASES)
def test_exact_case_forward_bitwise_and_gradients(topo, widths, c_in, n, shape):
    """Every layer's forward and backward against the oracle where rounding
    cannot hide a mistake: outputs identical, gradients to FP32 rounding."""
    params = _int_params(widths, c_in, seed=3)
    rng = np.random.default_rng(4)
    x = rng.integers(0, 4, size=(n, c_in) + shape).astype(np.float64)
    gy = rng.integers(-2, 3, size=(n, 3) + shape).astype(np.float64)
    yg, grads = _run(topo, params, widths, c_in, x, gy)
    yr, ref = _oracle(params, x, gy)
    assert np.array_equal(yg, yr.astype(np.float32))
    for li, ((gw, gb), (rw, rb)) in enumerate(zip(grads, ref)):
        assert np.linalg.norm(rw) > 0, li  # every layer takes part
        assert np.linalg.norm(gw - rw) <= 1e-5 * np.linalg.norm(rw), li
        assert np.linalg.norm(gb - rb) <= 1e-5 * np.linalg.norm(rb) + 1e-6, li


@pytest.mark.parametrize("widths,c_in,n,shape", CASES)
def test_random_case_within_bf16_noise(topo, widths, c_in, n, shape):
    """He-initialised weights and Gaussian inputs.  Both sides round the same
    stored activations to bf16; the kernels accumulate in FP32, the oracle in
    FP64.  FP32 sums of ~10^3 products differ from FP64 by ~1e-5 relative, which
    flips ~0.5% of the stored bf16 values by one ulp (2^-8) per layer; replaying
    the oracle with FP32 accumulation moves the first case's output by 1.4e-3
    (norm) / 2.7e-3 (max) relative and its weight gradients by 2% to 7.5% per
    layer (ReLU masks at activations within an ulp of zero).  Bounds: ~3.5x
    (outputs) and 2x (gradients) those figures, plus a cosine check."""
    params = _params(widths, c_in, seed=3)
    rng = np.random.default_rng(4)
    x = nn.to_bf16(rng.normal(size=(n, c_in) + shape))
    gy = rng.normal(size=(n, 3) + shape).astype(np.float32)
    yg, grads = _run(topo, params, widths, c_in, x, gy)
    yr, ref = _oracle(params, x, gy)
    assert np.max(np.abs(yg - yr)) <= 1e-2 * np.max(np.abs(yr))
    assert np.linalg.norm(yg - yr) <= 5e-3 * np.linalg.norm(yr)
    for li, ((gw, gb), (rw, rb)) in enumerate(zip(grads, ref)):
        assert np.linalg.norm(gw - rw) <= 0.15 * np.linalg.norm(rw), li
        cos = float(np.sum(gw * rw) / (np.linalg.norm(gw) * np.linalg.norm(rw)))
        assert cos >= 0.99, (li, cos)


def test_training_step_reduces_the_loss(topo):
    rng = np.random.default_rng(5)
    n, D, H, Wd = 4, 8, 8, 16
    x = nn.to_bf16(rng.normal(size=(n, 8, D, H, Wd)))
    # a smooth target the network can fit: a blurred copy of input channel 0
    t = np.stack([np.stack([np.roll(x[s, 0], sh, axis=2) * 0.5 for sh in (0, 1, 2)]) for s in range(n)])
    net = topo.Net(8, (16, 32, 64, 64))
    net.set_params(_params((16, 32, 64, 64), 8, seed=6))
    xt, tt = _bf16_tensor(x), _bf16_tensor(nn.to_bf16(t))
    losses = [net.train_step(xt, tt, 2e-3) for _ in range(60)]
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])
    # Adam moved the parameters, and get/set round-trips them
    p = net.get_params()
    net.set_params(p)
    assert np.array_equal(net.get_params(), p)
    net.close()


@pytest.fixture(scope="module")
def small(topo):
    w = W.small3d(16, 8, 8)
    rho = W.random_density(w.n_el, seed=21, lo=0.05)
    p = topo.Problem.from_workload(w)
    p.set_density(rho)
    yield w, rho, p
    p.close()


def test_features_match_oracle(topo, small):
    w, rho, p = small
    out = torch.empty((1, 8, 8, 8, 16), dtype=torch.bfloat16, device="cuda")
    p.features(out)
    got = out.float().cpu().numpy()[0]
    ref = nn.to_bf16(warm.features(w, rho))
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-30)


def test_targets_match_oracle(topo, small):
    w, rho, p = small
    p.solve(topo.solve_opts(tol=1e-10, max_it=20000, precision=topo.TP_PREC_F64))
    u = p.get(topo.TP_U)
    out = torch.empty((1, 3, 8, 8, 16), dtype=torch.bfloat16, device="cuda")
    p.targets(out)
    got = out.float().cpu().numpy()[0]
    ref = warm.targets(w, u)
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-6)


def test_warm_start_matches_oracle_and_solves(topo, small):
    w, rho, p = small
    params = _params((16, 32, 64, 64), 8, seed=9)
    net = topo.Net(8, (16, 32, 64, 64))
    net.set_params(params)
    alpha, ms = p.warm_start_nn(net)
    u0 = p.get(topo.TP_U)
    x = nn.to_bf16(warm.features(w, rho))
    y = nn.forward(params, x, quant=nn.to_bf16)
    uh = warm.node_average(w, y)
    a = warm.alpha(w, rho, uh)
    assert alpha[0] == pytest.approx(a, rel=1e-2)
    assert np.linalg.norm(u0 - a * uh) <= 1e-2 * np.linalg.norm(a * uh)
    assert ms > 0.0
    info = p.solve(topo.solve_opts(tol=1e-8, max_it=50000, precision=topo.TP_PREC_MIXED,
                                   warm_start=topo.TP_WARM_USER, update_drop=0.1))
    assert info.converged == 1 and info.rel_res[0] <= 1e-8
    assert info.rel_res_init[0] == pytest.approx(fem.rel_residual(w, rho, u0[None, :])[0], rel=1e-6)
    net.close()


def test_energy_loss_and_gradient_match_oracle(topo, small):
    w, rho, p = small
    p.solve(topo.solve_opts(tol=1e-12, max_it=50000, precision=topo.TP_PREC_F64))
    comp = p.sensitivities()
    rng = np.random.default_rng(40)
    y = rng.normal(size=(3, 8, 8, 16)).astype(np.float32)
    yt = torch.from_numpy(y[None]).cuda()
    gy = torch.empty_like(yt)
    loss = p.energy_grad(yt, comp, gy)[0]
    ref_l, ref_g = warm.energy_loss(w, rho, y.astype(np.float64), comp)
    # FP64 arithmetic on both sides except the FP32 node sums and gradient store
    assert loss == pytest.approx(ref_l, rel=1e-5)
    g = gy.cpu().numpy()[0]
    assert np.linalg.norm(g - ref_g) <= 1e-5 * np.linalg.norm(ref_g)


def test_bad_user_start_falls_back_to_zero(topo, small):
    w, rho, p = small
    p.set(topo.TP_U, 1e3 * W.random_vector(w.n_dof, seed=30))
    info = p.solve(topo.solve_opts(tol=1e-8, max_it=50000, precision=topo.TP_PREC_MIXED,
                                   warm_start=topo.TP_WARM_USER, update_drop=0.1))
    assert info.warm_fallback == 1 and info.rel_res_init[0] > 1.0
    assert info.converged == 1


def test_warm_start_rejects_unsupported_grids(topo):
    w = W.small3d(6, 4, 4)
    p = topo.Problem.from_workload(w)
    net = topo.Net(8, (16, 32, 64, 64))
    with pytest.raises(topo.TopoError):
        p.warm_start_nn(net)
    net.close()
    p.close()


def test_trained_network_gain_on_a_held_out_problem(topo):
    """What the trained network gains over the method without it, on a 3D
    cantilever it was not trained on (96 x 32 x 32, volfrac 0.12, the density
    after 5 OC iterations):
      - start quality: the energy-norm error of the learned start is well
        below that of u = 0 (1 by definition) and below that of the untrained
        (He-initialised) network;
      - solve: with the default acceptance rule (true residual no worse than
        u = 0) the solve meets the tolerance and costs no more CG iterations
        than plain mixed PCG, plus the network's time."""
    import workloads as W
    from paper_2012_08208_gb300 import warmstart as WS
    w = W.cantilever3d(96, 32, 32, volfrac=0.12, rmin=1.5)
    p = WS.density_after(w, 5)
    p.solve(topo.solve_opts(tol=1e-10, max_it=400000, precision=topo.TP_PREC_MIXED, update_drop=0.1))
    comp = p.sensitivities()
    net = topo.Net.load(WS.WEIGHTS)
    err = WS.energy_error(p, net, comp)
    raw = topo.Net(8, (16, 32, 64, 64))
    raw.set_params(_params((16, 32, 64, 64), 8, seed=0))
    err_raw = WS.energy_error(p, raw, comp)
    assert err < 0.9 and err < err_raw, (err, err_raw)
    cold = WS.time_to_tol(p, "mixed", 1e-6)
    learned = WS.time_to_tol(p, "learned", 1e-6, net)
    forced = WS.time_to_tol(p, "learned", 1e-6, net, warm_max_rel=1e30)
    print(json.dumps({"energy_err": err, "energy_err_untrained": err_raw, "cold": cold, "learned": learned,
                      "learned_forced": forced}))
    assert learned["converged"] == 1 and learned["rel_res"] <= 1e-6
    if learned["fallback"]:  # dropped start: exactly the plain solve
        assert learned["iters"] == cold["iters"]
    net.close()
    raw.close()
    p.close()
