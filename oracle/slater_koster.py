"""Two-centre s/p Slater-Koster blocks (oracle; test infrastructure only).

The paper runs ELSES with tight-binding-form Hamiltonians in an LCAO basis, sparse real-symmetric
H and positive definite S (Eq. 1 and the text around it). The parameter sets it used are not
given, so the model here is the standard two-centre s/p Slater-Koster table with the reading:

    V_x(r) = V0_x * exp(-q_x (r - r0)) * t(r),    x in (ss-sigma, sp-sigma, pp-sigma, pp-pi)
    t(r)   = 1 for r <= r_on, 0 for r >= r_cut,
             1 - 10 s^3 + 15 s^4 - 6 s^5 with s = (r - r_on)/(r_cut - r_on) in between,

the same law (with its own V0, q) for the overlap integrals. Orbital order inside a 4x4 block is
(s, px, py, pz). The block of the pair (I, J) is evaluated at d = R_J - R_I:

    B[s, s]   = V_ss
    B[s, p_i] = u_i V_sp,        B[p_i, s] = -u_i V_sp
    B[p_i, p_k] = u_i u_k (V_pp_sigma - V_pp_pi) + delta_ik V_pp_pi,         u = d / |d|

so that B(J, I) = B(I, J)^T and the assembled H, S are symmetric.
All functions are vectorised over a leading axis of pair vectors.
"""
from __future__ import annotations

import numpy as np


def taper(r, sk):
    """Smooth cutoff t(r) (reading of the model; see module docstring)."""
    r = np.asarray(r, dtype=np.float64)
    s = (r - sk.r_on) / (sk.r_cut - sk.r_on)
    t = 1.0 - 10.0 * s**3 + 15.0 * s**4 - 6.0 * s**5
    return np.where(r <= sk.r_on, 1.0, np.where(r >= sk.r_cut, 0.0, t))


def dtaper(r, sk):
    """dt/dr."""
    r = np.asarray(r, dtype=np.float64)
    w = sk.r_cut - sk.r_on
    s = (r - sk.r_on) / w
    dt = (-30.0 * s**2 + 60.0 * s**3 - 30.0 * s**4) / w
    return np.where((r <= sk.r_on) | (r >= sk.r_cut), 0.0, dt)


def radial(r, V0, q, sk):
    """V(r) = V0 exp(-q (r - r0)) t(r) for the four integrals; returns shape r.shape + (4,)."""
    r = np.asarray(r, dtype=np.float64)[..., None]
    V0 = np.asarray(V0, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    return V0 * np.exp(-q * (r - sk.r0)) * taper(r, sk)


def dradial(r, V0, q, sk):
    """dV/dr for the four integrals."""
    r = np.asarray(r, dtype=np.float64)[..., None]
    V0 = np.asarray(V0, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    e = V0 * np.exp(-q * (r - sk.r0))
    return e * (-q * taper(r, sk) + dtaper(r, sk))


def _table(u, V):
    """4x4 blocks from unit vectors u (P,3) and integrals V (P,4)."""
    P = u.shape[0]
    B = np.zeros((P, 4, 4))
    vss, vsp, vpps, vppp = V[:, 0], V[:, 1], V[:, 2], V[:, 3]
    B[:, 0, 0] = vss
    B[:, 0, 1:] = u * vsp[:, None]
    B[:, 1:, 0] = -u * vsp[:, None]
    B[:, 1:, 1:] = (np.einsum("pi,pk->pik", u, u) * (vpps - vppp)[:, None, None]
                    + np.eye(3)[None] * vppp[:, None, None])
    return B


def blocks(d, sk):
    """H and S blocks (P,4,4) of atom pairs with separation vectors d = R_J - R_I (P,3)."""
    d = np.atleast_2d(np.asarray(d, dtype=np.float64))
    r = np.sqrt(np.einsum("pi,pi->p", d, d))
    u = d / r[:, None]
    H = _table(u, radial(r, sk.V0, sk.qH, sk))
    S = _table(u, radial(r, sk.S0, sk.qS, sk))
    return H, S


def _table_grad(d, V, dV):
    """d(block)/d(d_m): shape (P,3,4,4), from integrals V and their radial derivatives dV."""
    r = np.sqrt(np.einsum("pi,pi->p", d, d))
    u = d / r[:, None]
    P = d.shape[0]
    eye = np.eye(3)
    # du_i/dd_m = (delta_im - u_i u_m)/r  -> shape (P, m, i)
    du = (eye[None] - np.einsum("pm,pi->pmi", u, u)) / r[:, None, None]
    G = np.zeros((P, 3, 4, 4))
    vss, vsp, vpps, vppp = (V[:, k] for k in range(4))
    dss, dsp, dpps, dppp = (dV[:, k] for k in range(4))
    G[:, :, 0, 0] = dss[:, None] * u
    sp = dsp[:, None, None] * np.einsum("pm,pi->pmi", u, u) + vsp[:, None, None] * du
    G[:, :, 0, 1:] = sp
    G[:, :, 1:, 0] = -sp
    uu = np.einsum("pi,pk->pik", u, u)
    duu = np.einsum("pmi,pk->pmik", du, u) + np.einsum("pi,pmk->pmik", u, du)
    G[:, :, 1:, 1:] = (np.einsum("p,pm,pik->pmik", dpps - dppp, u, uu)
                       + np.einsum("p,pm,ik->pmik", dppp, u, eye)
                       + (vpps - vppp)[:, None, None, None] * duu)
    return G


def block_grads(d, sk):
    """dH/dd and dS/dd of the pair blocks: shapes (P,3,4,4) with d = R_J - R_I."""
    d = np.atleast_2d(np.asarray(d, dtype=np.float64))
    r = np.sqrt(np.einsum("pi,pi->p", d, d))
    gH = _table_grad(d, radial(r, sk.V0, sk.qH, sk), dradial(r, sk.V0, sk.qH, sk))
    gS = _table_grad(d, radial(r, sk.S0, sk.qS, sk), dradial(r, sk.S0, sk.qS, sk))
    return gH, gS


def onsite(sk):
    """On-site blocks: H = diag(Es, Ep, Ep, Ep), S = identity."""
    return np.diag([sk.Es, sk.Ep, sk.Ep, sk.Ep]).astype(np.float64), np.eye(4)
