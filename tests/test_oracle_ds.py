"""Pins for the oracle's domain selection (Sec. III-B) and its generator."""

import math

import numpy as np
import pytest

import synth
from oracle import brute_force, ising, rng
from oracle import domain_selection as ds
from oracle import domain_selection as ods


def test_splitmix64_published_outputs():
    # SplitMix64 started at 0: first three outputs
    z = rng.splitmix64(0, np.arange(3))
    assert [int(x) for x in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                   0x06C45D188009454F]


def test_theta_init_relaxes_the_uniform_draw():
    x0 = rng.uniform_pm1(11, 8, 50)
    assert x0.min() >= -1.0 and x0.max() < 1.0
    assert abs(x0.mean()) < 0.15
    np.testing.assert_allclose(np.sin(rng.theta_init(11, 8, 50)), x0, atol=1e-15)


def _setup(seed=0, n=24, B=5, conv="physics"):
    inst = synth.random_sparse_instance(n, seed, p=0.3, kind="float", h="float",
                                        convention=conv, j_scale=0.5)
    cq, ch = ising.coefficients(inst.j_scale, inst.convention)
    J = ising.coupling_matrix(inst)
    h = ising.field(inst)
    theta = np.random.default_rng(seed).uniform(-math.pi, math.pi, (n, B))
    return inst, cq, ch, J, h, theta


@pytest.mark.parametrize("conv", ["physics", "paper"])
def test_gradient_matches_finite_difference(conv):
    inst, cq, ch, J, h, theta = _setup(conv=conv)
    p = ds.Params(mu=0.7)
    s = ds.round_spins(theta)
    r = ds.step(J, h, cq, ch, p, theta, np.zeros_like(theta), np.zeros_like(theta), 1)
    d = 1e-6
    for i in range(0, inst.n, 5):
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += d
        tm[i] -= d
        fd = (ds.loss(J, h, cq, ch, p.mu, tp, s) - ds.loss(J, h, cq, ch, p.mu, tm, s)) / (2 * d)
        np.testing.assert_allclose(r.grad[i], fd, rtol=1e-6, atol=1e-7)


def test_loss_at_the_corners_is_energy_minus_mu_d():
    # with |sin theta| = 1 the loss of Eq. (loss function) is s^T (A - mu I) s + b^T s
    inst, cq, ch, J, h, _ = _setup(n=18, B=4)
    s = (2 * np.random.default_rng(3).integers(0, 2, (18, 4)) - 1).astype(float)
    theta = s * (math.pi / 2)
    mu = 1.3
    L = ds.loss(J, h, cq, ch, mu, theta, ds.round_spins(theta))
    np.testing.assert_allclose(L, ising.energy(inst, s) - mu * 18, rtol=1e-12)


def test_adam_matches_torch_adam():
    torch = pytest.importorskip("torch")
    inst, cq, ch, J, h, theta = _setup(n=16, B=3)
    p = ds.Params(lr=0.05, mu=0.2, beta1=0.8, beta2=0.99, eps=1e-6)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([th], lr=p.lr, betas=(p.beta1, p.beta2), eps=p.eps)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    cur = theta.copy()
    for t in range(1, 6):
        r = ds.step(J, h, cq, ch, p, cur, m, v, t)
        # torch sees the same gradient of the frozen-spin loss at the same point
        with torch.no_grad():
            th.copy_(torch.tensor(cur))
        s = torch.tensor(ds.round_spins(cur))
        F = torch.tensor(r.F)
        opt.zero_grad()
        (torch.sin(th) * F).sum().backward()
        np.testing.assert_allclose(th.grad.numpy(), r.grad, rtol=1e-13, atol=1e-13)
        opt.step()
        ref = th.detach().numpy()
        diff = r.theta - ref
        diff -= 2 * math.pi * np.rint(diff / (2 * math.pi))
        assert np.max(np.abs(diff)) < 1e-12
        assert s is not None
        cur, m, v = r.theta, r.m, r.v


def test_first_step_moves_each_angle_by_lr():
    inst, cq, ch, J, h, theta = _setup(n=30, B=4)
    p = ds.Params(lr=0.3, mu=0.1)
    r = ds.step(J, h, cq, ch, p, theta, np.zeros_like(theta), np.zeros_like(theta), 1)
    moved = r.theta - theta
    moved -= 2 * math.pi * np.rint(moved / (2 * math.pi))
    big = np.abs(r.grad) > 1e-3
    np.testing.assert_allclose(np.abs(moved[big]), p.lr, rtol=1e-5)
    assert np.all(np.sign(moved[big]) == -np.sign(r.grad[big]))
    assert np.all(np.abs(r.theta) <= math.pi + 1e-12)


def test_sgn_plus_of_zero_is_plus_one():
    """sgn+(0) = +1 (the reading of the unspecified sign at 0): theta = 0 and
    -0 round to +1, and so does the initial draw x0 = 0 (theta = asin 0 = 0);
    just below 0 rounds to -1."""
    th = np.array([[0.0, -0.0, -1e-300, 1e-300]])
    np.testing.assert_array_equal(ds.round_spins(th), [[1.0, 1.0, -1.0, 1.0]])
    inst = synth.er_dense(6, 1, p=0.5, weights="pm1")
    cq, ch = ising.coefficients(inst.j_scale, inst.convention)
    J, h = ising.coupling_matrix(inst), ising.field(inst)
    r = ds.step(J, h, cq, ch, ds.Params(lr=0.1), np.zeros((6, 2)), np.zeros((6, 2)), np.zeros((6, 2)), 1)
    np.testing.assert_array_equal(r.spins, np.ones((6, 2)))
    np.testing.assert_array_equal(r.energy, ising.energy(inst, np.ones((6, 2))))


def test_projection_is_the_ieee_remainder_modulo_two_pi():
    """The projection onto the relaxed domain maps an angle to its IEEE
    remainder modulo 2 pi (math.remainder: theta - 2 pi k, k the nearest
    integer, result in [-pi, pi]). A first Adam step with lr = 6 from angles
    near +-pi moves each by lr sgn(g) |g| / (|g| + eps) (m-hat / sqrt(v-hat) =
    sgn g at t = 1), far outside [-pi, pi]; the oracle's result must be that
    move's remainder, computed here with the library routine."""
    inst, cq, ch, J, h, _ = _setup(n=20, B=3)
    r0 = np.random.default_rng(8)
    theta = np.where(r0.random((20, 3)) < 0.5, -1.0, 1.0) * r0.uniform(2.9, 3.1, (20, 3))
    p = ds.Params(lr=6.0, mu=0.05)
    r = ds.step(J, h, cq, ch, p, theta, np.zeros_like(theta), np.zeros_like(theta), 1)
    g = r.grad
    raw = theta - p.lr * np.sign(g) * np.abs(g) / (np.abs(g) + p.eps)
    want = np.vectorize(lambda x: math.remainder(x, 2 * math.pi))(raw)
    np.testing.assert_allclose(r.theta, want, rtol=0, atol=1e-12)
    assert np.all(np.abs(r.theta) <= math.pi)
    # sin and cos of the projected angle are those of the unprojected one
    np.testing.assert_allclose(np.sin(r.theta), np.sin(raw), atol=1e-12)
    np.testing.assert_allclose(np.cos(r.theta), np.cos(raw), atol=1e-12)


@pytest.mark.parametrize("trace,stop", [
    # E_1 = 10; windows 10..1 (spread 9), 5..1 (4), 3..1 (2), 2..1 (1) exceed
    # 0.005 |E_t - 10| = 0.045; the window of five 1s has spread 0: stop at t = 9
    ([10, 5, 3, 2, 1, 1, 1, 1, 1, 1], 9),
    # spread exactly at the tolerance stops (<=): E_1 = 0, E_t = -1000 from
    # t = 2 on except E_6 = -995; at t = 6 the spread 5 exceeds 0.005 |-995|
    # = 4.975, at t = 7 it equals 0.005 |-1000| = 5 and the restart stops
    ([0, -1000, -1000, -1000, -1000, -995, -1000, -1000], 7),
    # spread just above it does not stop until the 5.0001 leaves the window
    ([0, -1000, -1000, -1000, -1000, -994.9999, -1000, -1000, -1000, -1000, -1000], 11),
    # never converging: the energy keeps falling by 1 per step
    ([-t for t in range(12)], 0),
    # constant from the start: the window spread 0 <= 0 at t = 5
    ([-3.5] * 7, 5),
])
def test_convergence_rule_on_hand_computed_traces(trace, stop):
    """The Sec. IV-B stopping rule on energy traces whose stopping step is
    worked out by hand (the comments): window of 5, tolerance 0.005 of the
    change since the first step, inclusive comparison."""
    tr = np.asarray(trace, dtype=np.float64)
    got = 0
    for t in range(ds.CONV_WINDOW, len(tr) + 1):
        w = tr[t - ds.CONV_WINDOW:t][:, None]
        if ds.converged(w, tr[t - 1:t], tr[0:1])[0]:
            got = t
            break
    assert got == stop


def test_best_tracking_follows_the_trace():
    inst = synth.sk_dense(40, 2, 1.0)
    r = ds.select_domain(inst, ds.Params(restarts=6, steps=40, lr=0.3, seed=5), trace=True)
    tr = r["trace"]
    np.testing.assert_array_equal(r["restart_best_energy"], tr.min(axis=0))
    np.testing.assert_array_equal(r["restart_best_step"], tr.argmin(axis=0) + 1)
    # the stored best spins have the stored best energy
    np.testing.assert_allclose(ising.energy(inst, r["restart_best_spins"]),
                               r["restart_best_energy"], rtol=1e-12)
    assert r["best_energy"] == tr.min()
    assert r["best_restart"] == int(np.nonzero(tr.min(axis=0) == tr.min())[0][0])


@pytest.mark.parametrize("n", [16, 20])
def test_reaches_brute_force_ground_states(n):
    hits = 0
    for seed in range(4):
        inst = synth.sk_dense(n, 100 + seed, 1.0)
        e0, _ = brute_force.ground_state(inst)
        r = ds.select_domain(inst, ds.Params(restarts=64, steps=150, lr=6.0, seed=seed))
        assert r["best_energy"] >= e0 - 1e-9
        hits += abs(r["best_energy"] - e0) < 1e-9
    assert hits >= 3


def test_convergence_rule_closed_form_without_motion():
    """lr = 0 leaves theta where it starts: every restart's energy is the same
    at every step, the spread is 0 <= 0.005 |E_t - E_1| = 0, so all restarts
    stop at the fifth step and the run ends there (Sec. IV-B rule)."""
    inst = synth.er_dense(40, 2, p=0.2, weights="pm1")
    r = ods.select_domain(inst, ods.Params(restarts=6, steps=50, lr=0.0, seed=3), converge=True,
                          trace=True)
    assert (r["conv_step"] == ods.CONV_WINDOW).all() and r["steps_done"] == ods.CONV_WINDOW
    np.testing.assert_array_equal(r["restart_best_step"], 1)
    np.testing.assert_array_equal(r["restart_best_energy"], r["trace"][0])


@pytest.mark.parametrize("lr,h", [(0.05, None), (6.0, "int")])
def test_convergence_steps_follow_the_energy_trace(lr, h):
    """Against the trace of the same run without the rule (the dynamics do not
    depend on it): each restart stops at the first step where the window
    spread is within the tolerance, its best is the trace minimum up to
    there, and restarts that never stop keep the plain run's best."""
    inst = synth.random_sparse_instance(30, 5, p=0.3, kind="int", h=h or "none", layout="dense")
    p = ods.Params(restarts=12, steps=120, lr=lr, seed=7)
    plain = ods.select_domain(inst, p, trace=True)
    conv = ods.select_domain(inst, p, converge=True)
    tr = plain["trace"][:-1]  # E_1 .. E_T
    stops = 0
    for b in range(p.restarts):
        t_star = 0
        for t in range(ods.CONV_WINDOW, p.steps + 1):
            w = tr[t - ods.CONV_WINDOW:t, b]
            if w.max() - w.min() <= ods.CONV_TOL * abs(tr[t - 1, b] - tr[0, b]):
                t_star = t
                break
        assert conv["conv_step"][b] == t_star
        if t_star:
            stops += 1
            assert conv["restart_best_energy"][b] == tr[:t_star, b].min()
            assert conv["restart_best_step"][b] == int(np.argmin(tr[:t_star, b])) + 1
            assert conv["last_energy"][b] == tr[t_star - 1, b]
        else:
            assert conv["restart_best_energy"][b] == plain["restart_best_energy"][b]
    assert stops > 0


@pytest.mark.parametrize("conv", ["physics", "paper"])
def test_relaxed_gradient_matches_finite_difference(conv):
    """Relaxed product (G = J sin theta): the update direction cos(theta) F is
    the theta-gradient of cQ/2 x^T J x + cH h^T x - mu s^T x with s frozen;
    checked against central differences of that function computed directly
    from its definition (no oracle helper)."""
    inst = synth.random_sparse_instance(18, 3, p=0.4, kind="float", h="float",
                                       convention=conv, j_scale=0.5, layout="dense")
    cq, ch = ising.coefficients(inst.j_scale, inst.convention)
    J = ising.coupling_matrix(inst)
    h = ising.field(inst)
    mu = 0.3
    r = np.random.default_rng(5)
    theta = r.uniform(-3, 3, (18, 4))
    p = ds.Params(restarts=4, steps=1, lr=0.1, mu=mu, grad_mode="relaxed")
    res = ds.step(J, h, cq, ch, p, theta, np.zeros_like(theta), np.zeros_like(theta), 1)
    s = res.spins

    def f(th):
        x = np.sin(th)
        out = np.zeros(th.shape[1])
        for b in range(th.shape[1]):
            for i in range(th.shape[0]):
                out[b] += ch * h[i] * x[i, b] - mu * s[i, b] * x[i, b]
                for j in range(th.shape[0]):
                    out[b] += 0.5 * cq * J[i, j] * x[i, b] * x[j, b]
        return out

    eps = 1e-6
    for i in range(18):
        d = np.zeros_like(theta)
        d[i] = eps
        fd = (f(theta + d) - f(theta - d)) / (2 * eps)
        np.testing.assert_allclose(res.grad[i], fd, rtol=1e-6, atol=1e-7)
    # the energy reported is still that of the rounded spins
    np.testing.assert_allclose(res.energy, ising.energy(inst, s), rtol=1e-12)
    # at the corners (sin theta = s) the relaxed and rounded fields coincide
    corner = np.where(s > 0, np.pi / 2, -np.pi / 2)
    a = ds.step(J, h, cq, ch, p, corner, np.zeros_like(theta), np.zeros_like(theta), 1)
    b = ds.step(J, h, cq, ch, ds.Params(mu=mu), corner, np.zeros_like(theta), np.zeros_like(theta), 1)
    np.testing.assert_allclose(a.F, b.F, rtol=1e-12, atol=1e-12)
