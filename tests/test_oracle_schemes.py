"""Pins of the oracle's other time schemes (Remark "About the time
discretisation": a scheme changes Step 1 and the coefficient of M_H in Lambda).

- Heun's method on the 0-D Mitchell-Schaeffer cell against scipy's DOP853 at
  tight tolerance: second order (error ratio 4 per halving of the step).
- The reaction-free bidomain system (tau_in = tau_out = 1e300, so I_ion
  vanishes) has the exact solution V(t) = exp(-t/(chi Cm) M_H^-1 A) V(0) with
  A = S_i - S_i Pi S_1~^-1 Pi^T S_i (Prop. 2: K - gamma M_H) and U given by the
  elliptic equation: the semi-implicit Euler scheme of Sec. 3.2 converges at
  first order, Crank-Nicolson and Strang at second order, and Strang's U is
  the extracellular potential at the middle of the step.
- The full nonlinear schemes from a plateau state that never crosses the gate
  threshold (the gate's right-hand side is discontinuous there): Strang is
  second order; Euler and Crank-Nicolson with the reaction explicit at t^n are
  first order.
"""
import types

import numpy as np
from scipy.integrate import solve_ivp
from scipy.linalg import expm

from oracle import bidomain as ob
from oracle.algebra import pinv_psd
from workloads import torso_square_2d, params_2d

STEP = {"euler": ob.time_step, "cn": ob.time_step_cn, "strang": ob.time_step_strang}


def _ratios(errs):
    return [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]


def test_heun_is_second_order_on_the_cell():
    P = params_2d(0.1)
    span = P["v_peak"] - P["v_rest"]

    def f(t, y):
        i_ion, g = ob.ms_reaction(np.array([y[0]]), np.array([y[1]]), P)
        return [-i_ion[0] / P["Cm"], g[0]]

    y0 = [P["v_rest"] + 0.8 * span, 0.6]          # plateau: w stays above the gate
    ref = solve_ivp(f, (5.0, 15.0), y0, method="DOP853", rtol=1e-13, atol=1e-13).y[:, -1]
    cell = types.SimpleNamespace(params=P)
    errs = []
    for n in (100, 200, 400):
        v, h = np.array([y0[0]]), np.array([y0[1]])
        for k in range(n):
            v, h = ob.reaction_heun(cell, v, h, np.zeros(1), 5.0 + k * 10.0 / n, 5.0 + (k + 1) * 10.0 / n)
        errs.append(abs(v[0] - ref[0]))
    assert errs[-1] < 1e-6
    for r in _ratios(errs):
        assert 3.7 < r < 4.4, errs


def _diffusion_only():
    q = params_2d(0.1)
    q["tau_in"] = q["tau_out"] = 1e300       # I_ion = 0: the linear bidomain system
    q["chi"] = 10.0
    mesh = torso_square_2d(9)
    o = ob.build_system(mesh, q)
    N, NH = o.N, o.NH
    S1p, Si = pinv_psd(o.S1.toarray()), o.Si.toarray()
    Pi = np.eye(NH, N)
    A = Si - Si @ Pi @ S1p @ Pi.T @ Si

    def U_of(V):
        U = -S1p @ (Pi.T @ (Si @ V))
        return U - (o.M @ U).sum() / o.M.sum()

    xy = mesh.coords[o.order[:NH]]
    V0 = q["v_rest"] + 30.0 * np.exp(-((xy[:, 0] - 4.0) ** 2 + (xy[:, 1] - 5.0) ** 2) / 2.0)
    G = -np.diag(1.0 / o.MH.diagonal()) @ A / (q["chi"] * q["Cm"])
    return o, q, V0, U_of, lambda t: expm(t * G) @ V0


def test_diffusion_only_orders_against_the_matrix_exponential():
    o, q, V0, U_of, V_at = _diffusion_only()
    T, t0 = 4.0, 2.0                                 # stimulus off
    orders = {}
    for scheme, step in STEP.items():
        ev, eu = [], []
        for dt in (0.4, 0.2, 0.1):
            U, V, h = U_of(V0), V0.copy(), np.full(o.NH, 0.5)
            for k in range(int(round(T / dt))):
                U, V, h = step(o, U, V, h, np.zeros(o.NH), t0 + k * dt, dt)
            ev.append(np.abs(V - V_at(T)).max())
            # U of Euler and CN is at the step's end, Strang's at its middle
            u_ref = U_of(V_at(T - 0.5 * dt)) if scheme == "strang" else U_of(V_at(T))
            eu.append(np.abs(U - u_ref).max())
        orders[scheme] = (_ratios(ev), _ratios(eu))
    for r in orders["euler"][0]:
        assert 1.8 < r < 2.2, orders
    for scheme in ("cn", "strang"):
        for r in orders[scheme][0] + orders[scheme][1]:
            assert 3.7 < r < 4.4, (scheme, orders)


def test_full_schemes_self_convergence_from_a_plateau():
    q = params_2d(0.1)
    span = q["v_peak"] - q["v_rest"]
    mesh = torso_square_2d(13)
    o = ob.build_system(mesh, q)
    N, NH = o.N, o.NH
    S1p, Si = pinv_psd(o.S1.toarray()), o.Si.toarray()
    xy = mesh.coords[o.order[:NH]]
    V0 = q["v_rest"] + span * (0.6 + 0.2 * np.exp(-((xy[:, 0] - 4.0) ** 2 + (xy[:, 1] - 5.0) ** 2) / 2.0))
    U0 = -S1p @ (np.eye(NH, N).T @ (Si @ V0))
    U0 -= (o.M @ U0).sum() / o.M.sum()
    T, t0 = 2.0, 2.0
    for scheme, lo, hi in (("euler", 1.8, 2.3), ("cn", 1.8, 2.3), ("strang", 3.7, 4.4)):
        ends, wmin = [], 1.0
        for dt in (0.1, 0.05, 0.025):
            U, V, h = U0.copy(), V0.copy(), np.full(NH, 0.5)
            for k in range(int(round(T / dt))):
                U, V, h = STEP[scheme](o, U, V, h, np.zeros(NH), t0 + k * dt, dt)
                wmin = min(wmin, ((V - q["v_rest"]) / span).min())
            ends.append(V)
        assert wmin > q["v_gate"] + 0.1                # no gate switching on the way
        d = [np.abs(ends[0] - ends[1]).max(), np.abs(ends[1] - ends[2]).max()]
        assert lo < d[0] / d[1] < hi, (scheme, d)


def test_rest_is_a_fixed_point_of_every_scheme():
    mesh, q = torso_square_2d(13), params_2d(0.25)
    o = ob.build_system(mesh, q)
    U, V, h = ob.initial_state(o)
    for scheme, step in STEP.items():
        U1, V1, h1 = step(o, U, V, h, np.zeros(o.NH), 5.0, q["dt"])
        assert np.abs(V1 - q["v_rest"]).max() <= 1e-12 * abs(q["v_rest"]), scheme
        assert np.abs(U1).max() <= 1e-10 and np.array_equal(h1, h), scheme


def test_crank_nicolson_system_keeps_the_structure():
    # Lambda with 2 gamma: symmetric PSD with kernel [1; 0] exactly as for
    # gamma (Prop. 1); only the coefficient of M_H changes
    mesh, q = torso_square_2d(9), params_2d(0.25)
    o = ob.build_system(mesh, q)
    g = ob.gamma_of(q, q["dt"])
    assert ob.scheme_gamma(q, q["dt"], "euler") == g
    assert ob.scheme_gamma(q, q["dt"], "cn") == ob.scheme_gamma(q, q["dt"], "strang") == 2 * g
    L = ob.system_matrix(o, 2 * g).toarray()
    assert np.abs(L - L.T).max() == 0.0
    w, Q = np.linalg.eigh(L)
    assert np.abs(w[0]) <= 1e-12 * w[-1] and w[1] > 1e-8 * w[-1]
    k = Q[:, 0] / Q[0, 0]
    assert np.allclose(k[:o.N], 1.0) and np.abs(k[o.N:]).max() < 1e-10
