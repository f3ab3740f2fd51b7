"""Gradients of the multipole estimators with respect to the density mesh and to particle
positions (oracle; test infrastructure only).  Periodic box, global line of sight, one mesh with
mass-assignment compensation W(k) (no interlacing).

Forward quantities, from a real mesh delta(x) (index order x, y, z):
  X(q) = sum_x delta(x) e^{-i q.x} / W(q)
  P_l(b) = (2l+1)/(I22 N_b) sum_{q in b} L_l(qhat.los) |X(q)|^2 - delta_l0 N0          (Eq. Hand17)
  B_0(b) = sum_x F_b(x)^3 / (I33 sum_x I_b(x)^3),  F_b(x) = sum_{q in b} X(q) e^{i q.x}  (Eq. bi_sco,
           equilateral triangle (b, b, b))
with I22, I33, N0 held fixed (they depend on the catalogue, not on the mesh values).

Gradients (derived here; the paper gives none): for L = sum g_lb P_l(b) + sum h_b B_0(b),
  dL/ddelta(x) = sum_q [2 K(q) X(q) + sum_b c_b Phi_b(q) D_b(q)] / W(q) e^{i q.x}
  K(q) = sum_{l,b} g_lb (2l+1) Phi_b(q) L_l(qhat.los) / (I22 N_b),  c_b = 3 h_b / (I33 sum_x I_b^3),
  D_b(q) = sum_x F_b(x)^2 e^{-i q.x}.
TSC adjoint: delta(c) = sum_p w_p W3(c - s_p) (s = grid coordinate) gives
  dL/ds_p,a = w_p sum_c dL/ddelta(c) dW3/ds_a,  and dL/dx = (n/box) dL/ds.

Pinned by tests/test_oracle_adjoint.py with central finite differences of the forward functions.
"""
from __future__ import annotations

import numpy as np

from . import harmonics as H
from . import mesh as M


def _mu(n, box, los):
    (kx, ky, kz), _ = M.kvectors(n, box)
    d = np.asarray(los, dtype=np.float64)
    d = d / np.linalg.norm(d)
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(kk > 0, (kx * d[0] + ky * d[1] + kz * d[2]) / np.where(kk > 0, kk, 1.0), 0.0)


def spectrum(mesh, assign):
    n = mesh.shape[0]
    return np.fft.fftn(mesh) / M.window(n, assign)


def power_from_mesh(mesh, box, assign, kbins, ells, i22, n0, los=(0, 0, 1)):
    n = mesh.shape[0]
    X = spectrum(mesh, assign)
    b, _ = M.bin_index(n, box, *kbins)
    mu = _mu(n, box, los)
    out = {}
    for ell in ells:
        mean, cnt = M.bin_average(H.legendre(ell, mu) * np.abs(X) ** 2, b, kbins[2])
        out[ell] = np.where(cnt > 0, (2 * ell + 1) / i22 * mean - (n0 if ell == 0 else 0.0), 0.0)
    return out


def power_mesh_grad(mesh, box, assign, kbins, ells, i22, dldp, los=(0, 0, 1)):
    """dL/ddelta for L = sum_l sum_b dldp[l][b] P_l(b)."""
    n = mesh.shape[0]
    X = spectrum(mesh, assign)
    b, _ = M.bin_index(n, box, *kbins)
    mu = _mu(n, box, los)
    _, cnt = M.bin_average(np.zeros((n, n, n)), b, kbins[2])
    K = np.zeros((n, n, n))
    sel = b >= 0
    for ell in ells:
        g = np.asarray(dldp[ell], dtype=np.float64)
        coef = np.zeros(kbins[2])
        nz = cnt > 0
        coef[nz] = g[nz] * (2 * ell + 1) / (i22 * cnt[nz])
        K[sel] += coef[b[sel]] * H.legendre(ell, mu[sel])
    Y = 2.0 * K * X / M.window(n, assign)
    return np.real(np.fft.ifftn(Y)) * n**3


def _shells(X, n, box, kbins, ones=False):
    b, _ = M.bin_index(n, box, *kbins)
    out = []
    for ib in range(kbins[2]):
        mask = b == ib
        src = mask.astype(np.float64) if ones else np.where(mask, X, 0.0)
        out.append(np.real(np.fft.ifftn(src)) * n**3)
    return out


def bispec0_equilateral(mesh, box, assign, kbins, i33):
    n = mesh.shape[0]
    X = spectrum(mesh, assign)
    F = _shells(X, n, box, kbins)
    I = _shells(None, n, box, kbins, ones=True)
    return np.array([np.sum(F[k] ** 3) / (i33 * np.sum(I[k] ** 3)) if np.sum(I[k] ** 3) > 0 else 0.0
                     for k in range(kbins[2])])


def bispec0_mesh_grad(mesh, box, assign, kbins, i33, dldb):
    n = mesh.shape[0]
    X = spectrum(mesh, assign)
    F = _shells(X, n, box, kbins)
    I = _shells(None, n, box, kbins, ones=True)
    b, _ = M.bin_index(n, box, *kbins)
    Y = np.zeros((n, n, n), dtype=np.complex128)
    for k in range(kbins[2]):
        nt = np.sum(I[k] ** 3)
        if nt <= 0:
            continue
        c = 3.0 * dldb[k] / (i33 * nt)
        Y += np.where(b == k, c * np.fft.fftn(F[k] ** 2), 0.0)
    Y /= M.window(n, assign)
    return np.real(np.fft.ifftn(Y)) * n**3


def paint_tsc(s, w, n):
    return M.paint(s, w, n, 3)


def tsc_adjoint(s, w, grad_mesh):
    """dL/ds (npart, 3) for a TSC-painted mesh with cell gradient grad_mesh."""
    n = grad_mesh.shape[0]
    s = np.asarray(s, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    i0 = np.floor(s + 0.5)
    d = s - i0
    # weights and their derivatives with respect to s for taps -1, 0, +1 (d = s - i0)
    W = [0.5 * (0.5 - d) ** 2, 0.75 - d * d, 0.5 * (0.5 + d) ** 2]
    dW = [-(0.5 - d), -2.0 * d, (0.5 + d)]
    i0 = i0.astype(np.int64)
    out = np.zeros_like(s)
    for ox in range(3):
        ix = (i0[:, 0] + ox - 1) % n
        for oy in range(3):
            iy = (i0[:, 1] + oy - 1) % n
            for oz in range(3):
                iz = (i0[:, 2] + oz - 1) % n
                gv = grad_mesh[ix, iy, iz]
                out[:, 0] += gv * dW[ox][:, 0] * W[oy][:, 1] * W[oz][:, 2]
                out[:, 1] += gv * W[ox][:, 0] * dW[oy][:, 1] * W[oz][:, 2]
                out[:, 2] += gv * W[ox][:, 0] * W[oy][:, 1] * dW[oz][:, 2]
    return out * w[:, None]
