"""torch.autograd front end of the mesh-level estimators (include/npc.h, "Mesh-level estimators
and their adjoints"): argument marshalling only.  The forward values, the vector-Jacobian products
with respect to the mesh and the assignment adjoint with respect to particle positions and
weights all run in libnpc.so.

    mesh = paint(pos, w, n, box)                       # deterministic CIC/TSC assignment
    P, B0 = mesh_multipoles(mesh, box, kbins, ...)     # P_l (global LOS) and equilateral B_0
    (P[0] ** 2).sum().backward()                       # -> pos.grad, w.grad

Scope: periodic box, global line of sight, one mesh (no interlacing).
"""
from __future__ import annotations

import ctypes as C

import torch

from . import binding as B
from .api import _Keep, _prec, context, make_catalog, make_spec


def _dtype(precision):
    return torch.float64 if _prec(precision) == B.NPC_PREC_FP64 else torch.float32


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class _Cat:
    def __init__(self, pos, w):
        self.pos, self.w, self.nbar = pos, w, None


class PaintMesh(torch.autograd.Function):
    """pos [n,3], w [n] or None -> mesh [n,n,n] (index z, y, x) of the precision's dtype."""

    @staticmethod
    def forward(ctx, pos, w, n, box, origin, assign, precision):
        keep = _Keep()
        pos = pos.detach().contiguous()
        wd = w.detach().contiguous() if w is not None else None
        spec = make_spec(n, box, origin, assign, 0, 1, (0.0, 0.0, 1.0))
        cat = make_catalog(_Cat(pos, wd), keep)
        mesh = torch.empty((n, n, n), dtype=_dtype(precision), device=pos.device)
        h = context(pos.device.index or 0)
        B.check(B.npc_paint_mesh(h, C.byref(spec), C.byref(cat), _prec(precision), _ptr(mesh)), h)
        ctx.save_for_backward(pos, wd if wd is not None else torch.empty(0, device=pos.device))
        ctx.args = (n, box, tuple(origin), assign, precision, w is not None)
        return mesh

    @staticmethod
    def backward(ctx, gmesh):
        pos, wd = ctx.saved_tensors
        n, box, origin, assign, precision, has_w = ctx.args
        keep = _Keep()
        spec = make_spec(n, box, origin, assign, 0, 1, (0.0, 0.0, 1.0))
        cat = make_catalog(_Cat(pos, wd if has_w else None), keep)
        g = gmesh.to(_dtype(precision)).contiguous()
        gpos = torch.empty_like(pos)
        gw = torch.empty_like(wd) if has_w and ctx.needs_input_grad[1] else None
        h = context(pos.device.index or 0)
        B.check(B.npc_paint_adjoint(h, C.byref(spec), C.byref(cat), _ptr(g), _prec(precision), _ptr(gpos),
                                    _ptr(gw) if gw is not None else None), h)
        return gpos, gw, None, None, None, None, None


class MeshMultipoles(torch.autograd.Function):
    """mesh -> (P [nell, nbins], B0 [nbins], k_eff, N_modes, N_T); P and B0 are differentiable."""

    @staticmethod
    def forward(ctx, mesh, box, assign, los_dir, kbins, ells, b0, i22, n0, i33, precision):
        n = mesh.shape[0]
        assert mesh.shape == (n, n, n) and mesh.is_cuda and mesh.dtype == _dtype(precision)
        mesh = mesh.detach().contiguous()
        spec = make_spec(n, box, (0.0, 0.0, 0.0), assign, 0, 1, los_dir)
        kb = B.npc_kbins(float(kbins[0]), float(kbins[1]), int(kbins[2]))
        emask = sum(1 << int(l) for l in ells)
        length = int(B.npc_mesh_multipoles_len(C.byref(kb), emask, int(b0)))
        out = torch.zeros(max(length, 1), dtype=torch.float64, device=mesh.device)
        h = context(mesh.device.index or 0)
        B.check(B.npc_mesh_multipoles(h, C.byref(spec), _ptr(mesh), C.byref(kb), emask, int(b0), float(i22),
                                      float(n0), float(i33), _prec(precision), _ptr(out), 1), h)
        nb, ne = int(kbins[2]), len(ells)
        k_eff, nmodes = out[:nb], out[nb:2 * nb]
        P = out[2 * nb:(2 + ne) * nb].view(ne, nb).clone()
        if b0:
            B0 = out[(2 + ne) * nb:(3 + ne) * nb].clone()
            NT = out[(3 + ne) * nb:(4 + ne) * nb].clone()
        else:
            B0 = torch.zeros(0, dtype=torch.float64, device=mesh.device)
            NT = torch.zeros(0, dtype=torch.float64, device=mesh.device)
        ctx.save_for_backward(mesh)
        ctx.args = (box, assign, tuple(los_dir), tuple(kbins), tuple(ells), int(b0), float(i22), float(i33),
                    precision)
        k_eff, nmodes = k_eff.clone(), nmodes.clone()
        ctx.mark_non_differentiable(k_eff, nmodes, NT)
        return P, B0, k_eff, nmodes, NT

    @staticmethod
    def backward(ctx, gP, gB0, *_):
        (mesh,) = ctx.saved_tensors
        box, assign, los_dir, kbins, ells, b0, i22, i33, precision = ctx.args
        n = mesh.shape[0]
        spec = make_spec(n, box, (0.0, 0.0, 0.0), assign, 0, 1, los_dir)
        kb = B.npc_kbins(float(kbins[0]), float(kbins[1]), int(kbins[2]))
        emask = sum(1 << int(l) for l in ells)
        nb = int(kbins[2])
        dp = (gP if gP is not None else torch.zeros(len(ells), nb, device=mesh.device)).to(torch.float64).contiguous()
        db = None
        if b0:
            db = (gB0 if gB0 is not None else torch.zeros(nb, device=mesh.device)).to(torch.float64).contiguous()
        grad = torch.empty_like(mesh)
        h = context(mesh.device.index or 0)
        B.check(B.npc_mesh_multipoles_vjp(h, C.byref(spec), _ptr(mesh), C.byref(kb), emask, b0, i22, i33,
                                          _ptr(dp) if emask else None, _ptr(db) if b0 else None, 1,
                                          _prec(precision), _ptr(grad)), h)
        return grad, None, None, None, None, None, None, None, None, None, None


def paint(pos, w, n, box, origin=(0.0, 0.0, 0.0), assign=3, precision="mixed"):
    return PaintMesh.apply(pos, w, int(n), float(box), tuple(float(v) for v in origin), int(assign), precision)


def mesh_multipoles(mesh, box, kbins, ells=(0, 2, 4), b0=True, i22=1.0, n0=0.0, i33=1.0, assign=3,
                    los_dir=(0.0, 0.0, 1.0), precision="mixed"):
    """Returns dict(P=[nell, nbins], B0=[nbins], k_eff, nmodes, NT); P and B0 carry gradients."""
    P, B0, k_eff, nmodes, NT = MeshMultipoles.apply(mesh, float(box), int(assign), tuple(los_dir), tuple(kbins),
                                                    tuple(int(l) for l in ells), int(bool(b0)), i22, n0, i33,
                                                    precision)
    return {"P": P, "B0": B0, "k_eff": k_eff, "nmodes": nmodes, "NT": NT}


def periodic_normalisations(pos, w, box):
    """I22, N0, I33 of a periodic catalogue (float64 reductions in the library)."""
    from .api import catalog_scalars

    sc = catalog_scalars(_Cat(pos.detach(), None if w is None else w.detach()), None, box,
                         device=pos.device.index or 0)
    return sc["I22"], sc["N0"], sc["I33"]
