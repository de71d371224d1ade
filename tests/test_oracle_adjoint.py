"""Pins of the oracle's FP64 discrete adjoint (periodic D2Q4).

The adjoint is not in the paper; it is the transpose of the step the paper
defines.  Each pin checks it against finite differences of the oracle's own
forward map, which the other pin files tie to the paper:

  A1 equilibrium VJP:  <w, (E(U+hd) - E(U-hd))/2h>  ==  <J_E(U)^T w, d>
  A2 one adjoint step: <w, (step(fs+h d) - step(fs-h d))/2h> == <adjoint_step(w), d>
  A3 whole gradient of the config-5 style density loss over many steps against
     central differences along random directions and single entries.
  A4 at omega = 1 the adjoint of a step is the push of one 4-field quantity:
     dL/dfs^n_q(y) = (J_E(U(x))^T g(x))(x = y + c_q) for every q (the basis of the
     GPU sweep's 4-field form at omega = 1, as P2 is of the forward's moments-only form).
"""
import numpy as np
import pytest

import oracle
import workloads as W


def periodic(n, lam=3.0, omega=1.0):
    return oracle.Oracle(oracle.D2Q4, n, n, lam=lam, omega=omega, bc=[("periodic", None)] * 4)


def pulse_state(n, seed=0):
    wl, target = W.adjoint_pulses(seed=seed, n=n, pulses=3, width=0.15, steps=0)
    return wl.prim, target


def step(o, fs):
    f = o.stream(fs)
    fs1, U, _ = o.collide(f)
    return fs1, U


@pytest.mark.parametrize("omega", [1.0, 1.4])
def test_a1_equilibrium_vjp_matches_fd(omega):
    rng = np.random.default_rng(11)
    o = periodic(6, omega=omega)
    prim, _ = pulse_state(6)
    U = o.prim_to_cons(prim)
    w = rng.standard_normal((4, 4, 6, 6))
    d = rng.standard_normal((4, 6, 6))
    h = 1e-6
    lhs = np.sum(w * (o.feq(U + h * d) - o.feq(U - h * d)) / (2 * h))
    rhs = np.sum(o.vjp_equilibrium(U, w) * d)
    assert lhs == pytest.approx(rhs, rel=1e-8)


@pytest.mark.parametrize("omega", [1.0, 0.8, 1.6])
def test_a2_adjoint_step_is_transpose_of_step(omega):
    rng = np.random.default_rng(12)
    n = 8
    o = periodic(n, omega=omega)
    prim, _ = pulse_state(n, seed=1)
    fs = o.init(o.prim_to_cons(prim)) * (1 + 0.05 * rng.uniform(-1, 1, (4, 4, n, n)))
    _, U_next = step(o, fs)
    w = rng.standard_normal(fs.shape)
    d = rng.standard_normal(fs.shape)
    h = 1e-6
    jd = (step(o, fs + h * d)[0] - step(o, fs - h * d)[0]) / (2 * h)
    lhs = np.sum(w * jd)
    rhs = np.sum(o.adjoint_step(U_next, w) * d)
    assert lhs == pytest.approx(rhs, rel=1e-8)


def density_loss(o, fs, target, cell):
    rho = o.moments(fs)[0]
    return 0.5 * np.sum((rho - target) ** 2) * cell


@pytest.mark.parametrize("omega", [1.0, 1.3])
def test_a3_full_gradient_matches_central_differences(omega):
    n, steps = 16, 60
    o = periodic(n, omega=omega)
    prim, target = pulse_state(n, seed=2)
    U0 = o.prim_to_cons(prim)
    cell = (1.0 / n) ** 2

    def loss(U):
        fs, _ = o.run(o.init(U), steps)
        return density_loss(o, fs, target, cell)

    fs0, _ = o.run(o.init(U0), steps)
    dLdU = np.zeros((4, n, n))
    dLdU[0] = (o.moments(fs0)[0] - target) * cell
    grad, _ = o.gradient(U0, steps, dLdU)
    rng = np.random.default_rng(13)
    h = 1e-6
    for _ in range(4):
        d = rng.standard_normal(U0.shape)
        fd = (loss(U0 + h * d) - loss(U0 - h * d)) / (2 * h)
        assert np.sum(grad * d) == pytest.approx(fd, rel=1e-6)
    for _ in range(6):
        idx = tuple(rng.integers(0, s) for s in U0.shape)
        e = np.zeros_like(U0)
        e[idx] = 1.0
        fd = (loss(U0 + h * e) - loss(U0 - h * e)) / (2 * h)
        assert grad[idx] == pytest.approx(fd, rel=1e-5, abs=1e-12)


def test_adjoint_rejects_non_periodic():
    o = oracle.Oracle(oracle.D2Q4, 4, 4, lam=3.0, bc=[("transmissive", None)] * 4)
    with pytest.raises(ValueError):
        o.adjoint_step(np.ones((4, 4, 4)), np.ones((4, 4, 4, 4)))


def test_a4_omega1_adjoint_is_push_of_four_fields():
    rng = np.random.default_rng(14)
    n = 8
    o = periodic(n, omega=1.0)
    prim, _ = pulse_state(n, seed=2)
    fs = o.init(o.prim_to_cons(prim)) * (1 + 0.05 * rng.uniform(-1, 1, (4, 4, n, n)))
    _, U_next = step(o, fs)
    g = rng.standard_normal(fs.shape)
    out = o.adjoint_step(U_next, g)
    ubar = o.vjp_equilibrium(U_next, g)                 # J_E(U)^T g per cell: 4 fields
    SX, SY = [-1, 1, 1, -1], [-1, -1, 1, 1]
    for q in range(4):
        want = np.roll(ubar, shift=(-SY[q], -SX[q]), axis=(1, 2))   # ubar(y + c_q)
        assert np.allclose(out[q], want, rtol=1e-14, atol=1e-14 * np.abs(ubar).max())
    # and the 4-field form is not an identity of every omega
    o13 = periodic(n, omega=1.3)
    out13 = o13.adjoint_step(U_next, g)
    assert not np.allclose(out13[0], np.roll(o13.vjp_equilibrium(U_next, g), shift=(1, 1), axis=(1, 2)))

