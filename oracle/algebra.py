"""Dense matrices of Sec. 4 (tiny meshes only).  TEST INFRASTRUCTURE ONLY.

  pseudo-inverses S_1~^-1, S_i~^-1, S_e~^-1    Def. pseudo-inv
  K = gamma M_H + S_i - S_i Pi S_1~^-1 Pi^T S_i  Prop. 2, eq. LU2
  L, U with Lambda = L U                          Prop. 2, eq. LU
  L~^-1, U^-1                                     Prop. 3, eq. LU-inv
  harmonic-mean form of K                         Remark K
"""
from __future__ import annotations

import numpy as np

from .bidomain import System, restriction, monodomain_matrix


def pinv_psd(A: np.ndarray, rel: float = 1e-11) -> np.ndarray:
    """Pseudo-inverse of a symmetric PSD matrix: inverse on the range, zero on the
    kernel (eigenvalues below rel * max are taken as the kernel)."""
    w, V = np.linalg.eigh(A)
    keep = w > rel * w.max()
    return (V[:, keep] / w[keep]) @ V[:, keep].T


def dense_blocks(sys: System, gamma: float) -> dict:
    N, NH = sys.N, sys.NH
    Pi = restriction(N, NH).toarray()
    S1, Si, Se = sys.S1.toarray(), sys.Si.toarray(), sys.Se.toarray()
    MH = sys.MH.toarray()
    S1p, Sip, Sep = pinv_psd(S1), pinv_psd(Si), pinv_psd(Se)
    K = gamma * MH + Si - Si @ Pi @ S1p @ Pi.T @ Si
    Kinv = np.linalg.inv(K)
    I_N, I_H = np.eye(N), np.eye(NH)
    Z = np.zeros((N, NH))
    L = np.block([[S1, Z], [Si @ Pi, K]])
    U = np.block([[I_N, S1p @ Pi.T @ Si], [Z.T, I_H]])
    Lp = np.block([[S1p, Z], [-Kinv @ Si @ Pi @ S1p, Kinv]])
    Uinv = np.block([[I_N, -S1p @ Pi.T @ Si], [Z.T, I_H]])
    Lam = np.block([[S1, Pi.T @ Si], [Si @ Pi, gamma * MH + Si]])
    return dict(Pi=Pi, S1=S1, Si=Si, Se=Se, MH=MH, S1p=S1p, Sip=Sip, Sep=Sep, K=K,
                L=L, U=U, Lp=Lp, Uinv=Uinv, Lam=Lam,
                Km=monodomain_matrix(sys, gamma).toarray())


def harmonic_part_on_complement(blocks: dict):
    """Restrictions to 1_H^perp of K_0 = K - gamma M_H and of
    A = S_i~^-1 + Pi S_e~^-1 Pi^T (Remark K: K_0 = A^-1 there).
    Returns (Q^T K_0 Q, Q^T A Q) with Q an orthonormal basis of 1_H^perp."""
    NH = blocks["Si"].shape[0]
    one = np.ones((NH, 1)) / np.sqrt(NH)
    Qfull, _ = np.linalg.qr(np.hstack([one, np.eye(NH)[:, :NH - 1]]))
    Q = Qfull[:, 1:]
    Si, Pi = blocks["Si"], blocks["Pi"]
    K0 = Si - Si @ Pi @ blocks["S1p"] @ Pi.T @ Si
    A =blocks["Sip"] + blocks["Pi"] @ blocks["Sep"] @ blocks["Pi"].T
    return Q.T @ K0 @ Q, Q.T @ A @ Q
