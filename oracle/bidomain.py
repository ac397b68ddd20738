"""FP64 oracle: discretisation, scheme and solve of the bidomain time step.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Written from the paper:
  - tensors sigma_i, sigma_e (Sec. 2), sigma_1 and sigma_e-bar (Sec. 2.1, Rem. K),
    sigma_m = (sigma_e^-1 + sigma_i^-1)^-1 (Sec. 5.2);
  - matrices M, M_H, S_1, S_i defined by their bilinear forms (Sec. 3.1) with P1
    Lagrange elements and a lumped (row-sum) or consistent mass;
  - heart-first numbering so that Pi is a truncation (hypothesis H1, eq. def-Pi);
  - resolution algorithm, Steps 1-3 (Sec. 3.2), gamma = chi*Cm/dt;
  - Step 2 solved exactly on Ran(Lambda) and normalised (Prop. 1 and its proof).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# --------------------------------------------------------------------------
# P1 element quantities
# --------------------------------------------------------------------------

def p1_gradients(X: np.ndarray):
    """Barycentric gradients and measure of P1 simplices.

    X: (ne, d+1, d) vertex coordinates.  With J the matrix whose rows are the
    edge vectors x_k - x_0, a point is x = x_0 + J^T lambda, so the gradients of
    lambda_1..lambda_d are the rows of J^{-T}; grad lambda_0 = -sum of the others.
    Returns G (ne, d+1, d) and the element measures |det J| / d!.
    """
    d = X.shape[2]
    J = X[:, 1:, :] - X[:, :1, :]
    Jinv = np.linalg.inv(J)
    G = np.empty((X.shape[0], d + 1, d))
    G[:, 1:, :] = np.transpose(Jinv, (0, 2, 1))
    G[:, 0, :] = -G[:, 1:, :].sum(axis=1)
    vol = np.abs(np.linalg.det(J)) / (1.0 if d == 1 else (2.0 if d == 2 else 6.0))
    return G, vol


def element_stiffness(X: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    """K_e[i, j] = |e| * grad(l_i) . sigma grad(l_j) (sigma constant per element)."""
    G, vol = p1_gradients(X)
    return vol[:, None, None] * np.einsum("eia,eab,ejb->eij", G, sigma, G)


def element_mass(X: np.ndarray, lumped: bool) -> np.ndarray:
    """Consistent P1 mass |e|/((d+1)(d+2)) (1 + delta_ij), or its row sums."""
    _, vol = p1_gradients(X)
    d = X.shape[2]
    if lumped:
        m = np.zeros((X.shape[0], d + 1, d + 1))
        idx = np.arange(d + 1)
        m[:, idx, idx] = (vol / (d + 1))[:, None]
        return m
    base = (np.ones((d + 1, d + 1)) + np.eye(d + 1)) / ((d + 1) * (d + 2))
    return vol[:, None, None] * base[None]


def assemble(elems: np.ndarray, local: np.ndarray, n: int) -> sp.csr_matrix:
    """Sum element matrices into an n x n sparse matrix (duplicates are added)."""
    k = elems.shape[1]
    rows = np.repeat(elems, k, axis=1).ravel()
    cols = np.tile(elems, (1, k)).ravel()
    A = sp.coo_matrix((local.ravel(), (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def fibre_tensor(frames: np.ndarray, g: np.ndarray) -> np.ndarray:
    """sigma = F diag(g) F^T, F's columns being the local axes (Sec. 2)."""
    d = frames.shape[1]
    return np.einsum("eak,k,ebk->eab", frames, np.asarray(g[:d], dtype=np.float64), frames)


# --------------------------------------------------------------------------
# The discrete system (Sec. 3.1)
# --------------------------------------------------------------------------

@dataclass
class System:
    N: int
    NH: int
    order: np.ndarray        # new index -> mesh node
    new_of_old: np.ndarray   # mesh node -> new index
    S1: sp.csr_matrix
    Si: sp.csr_matrix
    Se: sp.csr_matrix
    Sm: sp.csr_matrix
    M: sp.csr_matrix
    MH: sp.csr_matrix
    params: dict


def heart_first_numbering(elems: np.ndarray, region: np.ndarray, n: int):
    """Heart nodes (vertices of heart elements) first, each group in mesh order."""
    heart = np.unique(elems[region == 1])
    is_heart = np.zeros(n, dtype=bool)
    is_heart[heart] = True
    order = np.concatenate([heart, np.nonzero(~is_heart)[0]])
    new_of_old = np.empty(n, dtype=np.int64)
    new_of_old[order] = np.arange(n)
    return order, new_of_old, int(heart.size)


def build_system(mesh, params: dict, lumped: bool = True) -> System:
    n = mesh.n_nodes
    order, new_of_old, NH = heart_first_numbering(mesh.elems, mesh.region, n)
    el = new_of_old[mesh.elems]                      # elements in the new numbering
    X = mesh.coords[mesh.elems]
    heart = mesh.region == 1
    d = mesh.dim
    sig_i = fibre_tensor(mesh.fibre, np.asarray(params["sigma_i"]))
    sig_e = fibre_tensor(mesh.fibre, np.asarray(params["sigma_e"]))
    iso = params["sigma_T"] * np.broadcast_to(np.eye(d), (mesh.n_elems, d, d))
    sig_1 = np.where(heart[:, None, None], sig_i + sig_e, iso)       # sigma_1 (Sec. 2.1)
    sig_eb = np.where(heart[:, None, None], sig_e, iso)              # sigma_e-bar (Rem. K)
    # sigma_m = (sigma_e^-1 + sigma_i^-1)^-1 on the heart (Sec. 5.2)
    sig_m = np.linalg.inv(np.linalg.inv(sig_e[heart]) + np.linalg.inv(sig_i[heart]))

    S1 = assemble(el, element_stiffness(X, sig_1), n)
    Se = assemble(el, element_stiffness(X, sig_eb), n)
    eh, Xh = el[heart], X[heart]
    Si = assemble(eh, element_stiffness(Xh, sig_i[heart]), NH)
    Sm = assemble(eh, element_stiffness(Xh, sig_m), NH)
    M = assemble(el, element_mass(X, lumped), n)
    MH = assemble(eh, element_mass(Xh, lumped), NH)
    return System(n, NH, order, new_of_old, S1, Si, Se, Sm, M, MH, dict(params))


def restriction(N: int, NH: int) -> sp.csr_matrix:
    """Pi: truncation of R^N to its first N_H entries (eq. def-Pi)."""
    return sp.eye(NH, N, format="csr")


def gamma_of(params: dict, dt: float) -> float:
    return params["chi"] * params["Cm"] / dt


def system_matrix(sys: System, gamma: float) -> sp.csr_matrix:
    """Lambda = [[S_1, Pi^T S_i], [S_i Pi, gamma M_H + S_i]] (eq. system)."""
    Pi = restriction(sys.N, sys.NH)
    return sp.bmat([[sys.S1, Pi.T @ sys.Si], [sys.Si @ Pi, gamma * sys.MH + sys.Si]],
                   format="csr")


def monodomain_matrix(sys: System, gamma: float) -> sp.csr_matrix:
    """K_m = gamma M_H + S_m (Sec. 5.2)."""
    return (gamma * sys.MH + sys.Sm).tocsr()


# --------------------------------------------------------------------------
# Reaction term: Mitchell-Schaeffer, in mV with w = (v - v_rest)/(v_peak - v_rest)
#   dw/dt = h w^2 (1 - w)/tau_in - w/tau_out,
#   dh/dt = (1 - h)/tau_open if w < v_gate else -h/tau_close,
#   Cm dv/dt = -I_ion  =>  I_ion = -Cm (v_peak - v_rest) (dw/dt without stimulus).
# --------------------------------------------------------------------------

def ms_reaction(v: np.ndarray, h: np.ndarray, p: dict):
    span = p["v_peak"] - p["v_rest"]
    w = (v - p["v_rest"]) / span
    j_in = h * w * w * (1.0 - w) / p["tau_in"]
    j_out = -w / p["tau_out"]
    i_ion = -p["Cm"] * span * (j_in + j_out)
    g = np.where(w < p["v_gate"], (1.0 - h) / p["tau_open"], -h / p["tau_close"])
    return i_ion, g


# --------------------------------------------------------------------------
# Step 2 solvers; all return X normalised so that int_Omega U = 0
# --------------------------------------------------------------------------

def normalise(sys: System, X: np.ndarray) -> np.ndarray:
    """U <- U - alpha 1 with alpha = (M U, 1)/(M 1, 1) (proof of Prop. 1)."""
    X = X.copy()
    U = X[:sys.N]
    one = np.ones(sys.N)
    alpha = (sys.M @ U).sum() / (sys.M @ one).sum()
    X[:sys.N] = U - alpha
    return X


def pinned_index(sys: System) -> int:
    """The U unknown fixed to zero in the pinned factorisations: the last node of
    the U block (the last torso node, or the last node of an isolated heart)."""
    return sys.N - 1


def solve_direct(sys: System, gamma: float, Y: np.ndarray) -> np.ndarray:
    """Exact solve for Y in Ran(Lambda): drop the pinned U unknown and its equation
    (the dropped equation is implied because the U block of Y sums to zero),
    solve the remaining SPD system with a sparse direct factorisation, then
    normalise."""
    L = system_matrix(sys, gamma)
    k = pinned_index(sys)
    keep = np.ones(L.shape[0], dtype=bool)
    keep[k] = False
    A = L[keep][:, keep].tocsc()
    X = np.zeros(L.shape[0])
    X[keep] = spla.spsolve(A, Y[keep])
    return normalise(sys, X)


def solve_cg(sys: System, gamma: float, Y: np.ndarray, X0=None, tol: float = 1e-13,
             max_iter: int = 200000):
    """Plain (unpreconditioned) CG on Lambda; the U block of the residual is
    projected onto 1^perp (Euclidean) after every update so that r stays in
    Ran(Lambda).  Stops on ||r||_2 / ||Y||_2 <= tol.  Returns (X, iterations)."""
    L = system_matrix(sys, gamma)
    N = sys.N
    x = np.zeros_like(Y) if X0 is None else np.array(X0, dtype=np.float64)
    ny = np.linalg.norm(Y)
    if ny == 0.0:
        return np.zeros_like(Y), 0
    r = Y - L @ x
    r[:N] -= r[:N].mean()
    p = r.copy()
    rho = r @ r
    it = 0
    while np.sqrt(rho) > tol * ny and it < max_iter:
        q = L @ p
        a = rho / (p @ q)
        x += a * p
        r -= a * q
        r[:N] -= r[:N].mean()
        rho_new = r @ r
        p = r + (rho_new / rho) * p
        rho = rho_new
        it += 1
    return normalise(sys, x), it


def solve_dense(sys: System, gamma: float, Y: np.ndarray) -> np.ndarray:
    """Dense symmetric pseudo-inverse (tiny meshes only), then normalisation."""
    L = system_matrix(sys, gamma).toarray()
    w, V = np.linalg.eigh(L)
    keep = np.abs(w) > 1e-12 * np.abs(w).max()
    X = V[:, keep] @ ((V[:, keep].T @ Y) / w[keep])
    return normalise(sys, X)


# --------------------------------------------------------------------------
# Resolution algorithm (Sec. 3.2)
# --------------------------------------------------------------------------

def stimulus_on(t: float, params: dict) -> bool:
    t0, t1 = params["stim_t"]
    return t0 <= t < t1


def rhs(sys: System, V: np.ndarray, h: np.ndarray, ist: np.ndarray, t: float, dt: float):
    """Step 1: Y = [0; M_H (gamma V^n - chi (I_ion(V^n, W^n) - I_st^n))]."""
    p = sys.params
    gamma = gamma_of(p, dt)
    i_ion, _ = ms_reaction(V, h, p)
    i_st = ist if stimulus_on(t, p) else np.zeros_like(V)
    y2 = sys.MH @ (gamma * V - p["chi"] * (i_ion - i_st))
    return np.concatenate([np.zeros(sys.N), y2])


def gate_update(sys: System, V: np.ndarray, h: np.ndarray, dt: float) -> np.ndarray:
    """Step 3: forward Euler on dW/dt = g(V, W), explicit in (V^n, W^n)."""
    _, g = ms_reaction(V, h, sys.params)
    return h + dt * g


def heart_stimulus(sys: System, node_amp: np.ndarray) -> np.ndarray:
    """Per-heart-node stimulus amplitude (new numbering) from a per-mesh-node one."""
    return np.asarray(node_amp, dtype=np.float64)[sys.order[:sys.NH]]


def initial_state(sys: System):
    """U = 0, V = v_rest, h = 1."""
    p = sys.params
    return np.zeros(sys.N), np.full(sys.NH, p["v_rest"]), np.ones(sys.NH)


def time_step(sys: System, U, V, h, ist, t: float, dt: float, solver: str = "direct",
              tol: float = 1e-13):
    """One step of the resolution algorithm; returns (U, V, h) at t + dt."""
    gamma = gamma_of(sys.params, dt)
    Y = rhs(sys, V, h, ist, t, dt)
    if solver == "direct":
        X = solve_direct(sys, gamma, Y)
    elif solver == "cg":
        X, _ = solve_cg(sys, gamma, Y, np.concatenate([U, V]), tol=tol)
    elif solver == "dense":
        X = solve_dense(sys, gamma, Y)
    else:
        raise ValueError(solver)
    h_new = gate_update(sys, V, h, dt)
    return X[:sys.N], X[sys.N:], h_new


# --------------------------------------------------------------------------
# Preconditioner at its exact limit (Def. 5.1, eq. prec2) with P_1 = S_1, P_K = K_m
# --------------------------------------------------------------------------

def s1_pseudo_inverse_apply(sys: System, b: np.ndarray) -> np.ndarray:
    """S_1-tilde^-1 b (Def. pseudo-inverse): project b onto 1^perp, solve with the
    pinned unknown removed, then project the result onto 1^perp."""
    b = b - b.mean()
    k = pinned_index(sys)
    keep = np.ones(sys.N, dtype=bool)
    keep[k] = False
    A = sys.S1[keep][:, keep].tocsc()
    x = np.zeros(sys.N)
    x[keep] = spla.spsolve(A, b[keep])
    return x - x.mean()


def precond_apply_exact(sys: System, gamma: float, r: np.ndarray) -> np.ndarray:
    """z = U_P^-1 L_P^-1 r with P_1 = S_1 (pseudo-inverse) and P_K = K_m."""
    N, NH = sys.N, sys.NH
    rU, rV = r[:N], r[N:]
    z1 = s1_pseudo_inverse_apply(sys, rU)
    t = rV - sys.Si @ z1[:NH]
    z2 = spla.spsolve(monodomain_matrix(sys, gamma).tocsc(), t)
    w = np.zeros(N)
    w[:NH] = sys.Si @ z2
    z1 = z1 - s1_pseudo_inverse_apply(sys, w)
    return np.concatenate([z1, z2])


# --------------------------------------------------------------------------
# Other time schemes (Remark "About the time discretisation"): a scheme
# changes the right-hand side of Step 1 and the coefficient of M_H in Lambda
# (hence in K); Lambda keeps its structure (symmetric PSD, kernel [1; 0]).
# Both schemes below treat the diffusion by Crank-Nicolson, so Lambda carries
# 2 gamma = 2 chi Cm / dt.
# --------------------------------------------------------------------------

def scheme_gamma(params: dict, dt: float, scheme: str) -> float:
    """Coefficient of M_H in Lambda: gamma (semi-implicit Euler, Sec. 3.2) or
    2 gamma (Crank-Nicolson diffusion, in the "cn" and "strang" schemes)."""
    g = gamma_of(params, dt)
    return g if scheme == "euler" else 2.0 * g


def rhs_cn(sys: System, U, V, h, ist, t: float, dt: float):
    """Step 1 of the Crank-Nicolson scheme, reaction explicit at t^n.  The
    parabolic equation averaged between t^n and t^n+1,
      chi Cm M_H (V' - V)/dt + chi M_H (I_ion - I_st)
          = -1/2 S_i (Pi U' + V') - 1/2 S_i (Pi U + V),
    with the elliptic equation S_1 U' + Pi^T S_i V' = 0 at t^n+1, is
    Lambda(2 gamma) X' = [0; M_H (2 gamma V - 2 chi (I_ion - I_st)) - S_i (Pi U + V)]."""
    p = sys.params
    g = gamma_of(p, dt)
    i_ion, _ = ms_reaction(V, h, p)
    i_st = ist if stimulus_on(t, p) else np.zeros_like(V)
    y2 = sys.MH @ (2.0 * g * V - 2.0 * p["chi"] * (i_ion - i_st)) - sys.Si @ (U[:sys.NH] + V)
    return np.concatenate([np.zeros(sys.N), y2])


def reaction_heun(sys: System, V, h, ist, t0: float, t1: float):
    """The reaction ODEs  Cm dv/dt = -(I_ion(v, h) - I_st(t)),  dh/dt = g(v, h)
    at every heart node over [t0, t1] by Heun's method (explicit trapezoidal
    rule, second order): with tau = t1 - t0, k1 = F(y, t0),
    k2 = F(y + tau k1, t1), y <- y + tau (k1 + k2)/2."""
    p = sys.params
    tau, t = t1 - t0, t0

    def F(v, hh, tt):
        i_ion, gg = ms_reaction(v, hh, p)
        i_st = ist if stimulus_on(tt, p) else np.zeros_like(v)
        return -(i_ion - i_st) / p["Cm"], gg

    dv1, dh1 = F(V, h, t)
    dv2, dh2 = F(V + tau * dv1, h + tau * dh1, t1)
    return V + 0.5 * tau * (dv1 + dv2), h + 0.5 * tau * (dh1 + dh2)


def _solve(sys: System, gamma: float, Y, X0, solver: str, tol: float):
    if solver == "direct":
        return solve_direct(sys, gamma, Y)
    if solver == "cg":
        return solve_cg(sys, gamma, Y, X0, tol=tol)[0]
    if solver == "dense":
        return solve_dense(sys, gamma, Y)
    raise ValueError(solver)


def time_step_cn(sys: System, U, V, h, ist, t: float, dt: float, solver: str = "direct",
                 tol: float = 1e-13):
    """One step of the Crank-Nicolson scheme (rhs_cn): returns (U, V, h) at
    t + dt; U must satisfy the elliptic equation with V (it does after any
    step, and for the resting initial state).  The gate takes its explicit
    Euler step from (V^n, W^n), as in Step 3."""
    Y = rhs_cn(sys, U, V, h, ist, t, dt)
    X = _solve(sys, scheme_gamma(sys.params, dt, "cn"), Y, np.concatenate([U, V]), solver, tol)
    return X[:sys.N], X[sys.N:], gate_update(sys, V, h, dt)


def time_step_strang(sys: System, U, V, h, ist, t: float, dt: float, solver: str = "direct",
                     tol: float = 1e-13):
    """One step of Strang splitting, reaction half step / diffusion step /
    reaction half step.  The reaction half steps are reaction_heun over
    [t, t + dt/2] and [t + dt/2, t + dt].  The diffusion step is
    Crank-Nicolson on the reaction-free bidomain system from V*: its midpoint
    Z = (X* + X')/2 solves Lambda(2 gamma) Z = [0; 2 gamma M_H V*] (the
    elliptic equation holds at both ends, so it holds for Z), and
    V' = 2 Z_V - V*.  The returned U is Z_U, the extracellular potential at
    the middle of the step, t + dt/2 (U at the step's end would need one more
    elliptic solve).  Returns (U_mid, V, h) with V and h at t + dt."""
    p = sys.params
    mid = t + 0.5 * dt
    Vs, hs = reaction_heun(sys, V, h, ist, t, mid)
    g2 = scheme_gamma(p, dt, "strang")
    Y = np.concatenate([np.zeros(sys.N), sys.MH @ (g2 * Vs)])
    Z = _solve(sys, g2, Y, np.concatenate([U, Vs]), solver, tol)
    V2 = 2.0 * Z[sys.N:] - Vs
    V3, h3 = reaction_heun(sys, V2, hs, ist, mid, t + dt)
    return Z[:sys.N], V3, h3
