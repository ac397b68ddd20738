"""Pins of the oracle's Mitchell-Schaeffer reaction term (workload input model,
Sec. 6.1 uses Luo-Rudy II instead) against the model's published closed forms."""
import numpy as np

from oracle import bidomain as ob
from workloads import params_2d


P = params_2d(0.25)


def test_rest_state_is_equilibrium():
    i_ion, g = ob.ms_reaction(np.array([P["v_rest"]]), np.array([1.0]), P)
    assert i_ion[0] == 0.0 and g[0] == 0.0


def test_gate_forward_euler_matches_exponential():
    # with v held fixed, h relaxes exponentially: to 1 with tau_open below the
    # gate, to 0 with tau_close above it; forward Euler is its first-order step
    dt = 0.01
    for v, tau, target in ((P["v_rest"] + 1.0, P["tau_open"], 1.0),
                           (P["v_peak"] - 1.0, P["tau_close"], 0.0)):
        h = np.array([0.4])
        _, g = ob.ms_reaction(np.array([v]), h, P)
        fe = h + dt * g
        exact = target + (h - target) * np.exp(-dt / tau)
        assert abs(fe - exact)[0] <= 0.5 * (dt / tau) ** 2 * abs(h - target)[0] * 1.01


def test_current_signs():
    # inward (negative) current in the upstroke range, outward just above rest
    v_mid = np.array([P["v_rest"] + 0.5 * (P["v_peak"] - P["v_rest"])])
    v_low = np.array([P["v_rest"] + 0.01 * (P["v_peak"] - P["v_rest"])])
    assert ob.ms_reaction(v_mid, np.array([1.0]), P)[0][0] < 0
    assert ob.ms_reaction(v_low, np.array([1.0]), P)[0][0] > 0


def test_action_potential_duration_closed_form():
    # 0-D cell: APD ~ tau_close * ln(tau_out / (4 tau_in)) (Mitchell & Schaeffer 2003)
    dt = 0.005
    v, h = np.array([P["v_rest"]]), np.array([1.0])
    span = P["v_peak"] - P["v_rest"]
    t, up, down = 0.0, None, None
    while t < 500.0:
        i_ion, g = ob.ms_reaction(v, h, P)
        ist = 50.0 if t < 1.0 else 0.0
        v = v + dt * (-(i_ion) + ist) / P["Cm"]
        h = h + dt * g
        t += dt
        w = (v[0] - P["v_rest"]) / span
        if up is None and w > 0.5:
            up = t
        if up is not None and down is None and w < 0.5 and t > up + 5:
            down = t
    apd = P["tau_close"] * np.log(P["tau_out"] / (4 * P["tau_in"]))
    assert up is not None and up < 3.0
    assert down is not None
    assert abs((down - up) - apd) < 0.1 * apd
