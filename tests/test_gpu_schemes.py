"""GPU parity of the Crank-Nicolson and Strang-splitting time schemes (the
paper's remark on the time discretisation) against the oracle's
time_step_cn / time_step_strang.

Per step the oracle is fed the GPU's state and takes the same step with a
sparse direct solve; the GPU solves to relative residual 1e-14.  U and V are
compared potential by potential within 1e-9 of the oracle block's largest
entry (as in test_gpu_parity), the gate h within 1e-13.  For Strang, U is the
extracellular potential at the middle of the step on both sides.
"""
import numpy as np
import pytest

from oracle import bidomain as ob
from potentials import assert_potentials_close
from workloads import torso_square_2d, slab_3d, params_2d, params_3d, stimulus_left_apex, \
    stimulus_centre_ball

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DEV = torch.device("cuda:0")
ORACLE_STEP = {"cn": ob.time_step_cn, "strang": ob.time_step_strang}


@pytest.fixture(scope="module")
def bid():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1711_08708_gb300 import bid as b
    return b


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def H(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("scheme", ["cn", "strang"])
def test_slice_steps_match_oracle(bid, scheme):
    # the 65^2 torso slice, dt 0.25 ms, corner stimulus (on for the first four
    # steps), 12 steps through the upstroke: the oracle fed the GPU's state
    # every step, and the two trajectories run apart agree at the end
    mesh, p = torso_square_2d(65), params_2d(0.25)
    S = bid.System(mesh, p)
    P = bid.Precond(S, p["dt"], eps=1e-3, precision="fp32", scheme=scheme)
    o = ob.build_system(mesh, p)
    assert (S.perm == o.order).all()
    ist = ob.heart_stimulus(o, stimulus_left_apex(mesh))
    U0, V0, h0 = ob.initial_state(o)
    U, V, h, I = T(U0), T(V0), T(h0), T(ist)
    Uo, Vo, ho = U0.copy(), V0.copy(), h0.copy()
    dt = p["dt"]
    for k in range(12):
        Ug, Vg, hg = H(U), H(V), H(h)
        its = P.step(U, V, h, I, k * dt, 1, tol=1e-14, max_iter=600)
        U1, V1, h1 = ORACLE_STEP[scheme](o, Ug, Vg, hg, ist, k * dt, dt)
        assert_potentials_close(np.concatenate([H(U), H(V)]), np.concatenate([U1, V1]), o.N, 1e-9,
                                (scheme, k))
        assert np.abs(H(h) - h1).max() <= 1e-13, (scheme, k)
        assert its[0] >= 1
        Uo, Vo, ho = ORACLE_STEP[scheme](o, Uo, Vo, ho, ist, k * dt, dt)
    assert_potentials_close(np.concatenate([H(U), H(V)]), np.concatenate([Uo, Vo]), o.N, 1e-9,
                            (scheme, "end"))
    assert np.abs(H(h) - ho).max() <= 1e-12
    assert H(V).max() > -60.0                 # the stimulus excited the corner


@pytest.mark.parametrize("scheme", ["cn", "strang"])
def test_slab_steps_match_oracle(bid, scheme):
    # isolated heart (Pi = Id): two steps of the small orthotropic slab
    mesh, p = slab_3d(13, 11, 7), params_3d(0.05)
    S = bid.System(mesh, p)
    P = bid.Precond(S, p["dt"], eps=0.0, scheme=scheme)
    o = ob.build_system(mesh, p)
    ist = ob.heart_stimulus(o, stimulus_centre_ball(mesh, radius=0.2))
    U0, V0, h0 = ob.initial_state(o)
    U, V, h, I = T(U0), T(V0), T(h0), T(ist)
    for k in range(2):
        Ug, Vg, hg = H(U), H(V), H(h)
        P.step(U, V, h, I, k * p["dt"], 1, tol=1e-14, max_iter=400)
        U1, V1, h1 = ORACLE_STEP[scheme](o, Ug, Vg, hg, ist, k * p["dt"], p["dt"])
        assert_potentials_close(np.concatenate([H(U), H(V)]), np.concatenate([U1, V1]), o.N, 1e-9,
                                (scheme, k))
        assert np.abs(H(h) - h1).max() <= 1e-13


def test_scheme_gamma_and_rejections(bid):
    # Crank-Nicolson doubles the coefficient of M_H: a CN preconditioner at dt
    # solves the same system as a semi-implicit one at dt / 2
    mesh, p = torso_square_2d(33), params_2d(0.1)
    S = bid.System(mesh, p)
    Pc = bid.Precond(S, 0.1, eps=0.0, scheme="cn")
    Pe = bid.Precond(S, 0.05, eps=0.0)
    o = ob.build_system(mesh, p)
    Y = ob.rhs(o, p["v_rest"] + 100 * np.random.default_rng(1).random(o.NH), np.ones(o.NH),
               np.zeros(o.NH), 5.0, 0.05)
    Xc = torch.zeros(o.N + o.NH, dtype=torch.float64, device=DEV)
    Xe = torch.zeros_like(Xc)
    ic = Pc.solve(T(Y), Xc, tol=1e-12)
    ie = Pe.solve(T(Y), Xe, tol=1e-12)
    assert ic["iters"] == ie["iters"]
    xc, xe = H(Xc), H(Xe)
    assert np.abs(xc - xe).max() <= 1e-12 * np.abs(xe).max()
    with pytest.raises(bid.BidError) as e:
        bid.Precond(S, 0.1, scheme=7)
    assert e.value.code == bid.EINVAL
    with pytest.raises(bid.BidError) as e:
        bid.Batch([S], 0.1, scheme="cn")
    assert e.value.code == bid.EINVAL
