"""Reverse mode of the coupled step for PyTorch: checkpointed recomputation
around the library's discrete adjoint (lbm_adjoint_step / lbm_adjoint_init).

``coupled_run(phi0, theta, case, nsteps, ckpt_every)`` advances one case (FP64
or FP32) and returns phi at the final step as a CUDA tensor; it is differentiable with
respect to the initial field phi0 and theta = (sigma, tau_g, lambda, tau_f) or,
for a case with walls, (sigma, tau_g, lambda, tau_f, u_wall_top, u_wall_bottom).
The forward pass records the states of the last steps in device memory, as
many as ``store_bytes`` holds (by default a quarter of the free device
memory), and a checkpoint every ``ckpt_every`` steps before them.  The
backward pass runs the adjoint steps straight from the recorded states; below
them it restores each checkpoint, recomputes the states of its segment and
runs the segment backwards.  So a run that fits in memory is differentiated
without recomputation.  All arithmetic runs in the CUDA library; torch holds
the device buffers.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbm


class AdjointSim:
    """One case with device snapshots and reverse-mode scratch.  Under FP32
    the states, adjoints and adjoint arithmetic are FP32 (the parameter
    derivatives accumulate in FP64); a snapshot has a 21st plane (the low
    part of the g_0 float pair)."""

    def __init__(self, case, phi0, u0=None, precision="f64"):
        self.case = dict(case)
        self.precision = precision
        self.dtype = torch.float64 if precision == "f64" else torch.float32
        self.sim = lbm.Sim(case, phi0, u0, precision=precision)
        self.h = self.sim.h
        self.dev = self.sim.device
        ny, nx = case["ny"], case["nx"]
        self.shape = (ny, nx)
        self.planes = lbm.lbm_snapshot_bytes(self.h, 0) // (self.dtype.itemsize * nx * ny)
        nb = lbm.lbm_adjoint_workspace_bytes(self.h)
        self._scratch = torch.empty(nb + 256, dtype=torch.uint8, device=self.dev)
        ptr = (self._scratch.data_ptr() + 255) // 256 * 256
        lbm.lbm_adjoint_attach(self.h, ptr, nb)
        self.phi0 = torch.as_tensor(np.ascontiguousarray(phi0), dtype=torch.float64,
                                    device=self.dev)
        self.u0 = None if u0 is None else torch.as_tensor(np.ascontiguousarray(u0),
                                                          dtype=torch.float64, device=self.dev)

    def new_state(self):
        return torch.zeros((20,) + self.shape, dtype=self.dtype, device=self.dev)

    def snapshot(self, buf=None):
        if buf is None:
            buf = torch.empty((self.planes,) + self.shape, dtype=self.dtype, device=self.dev)
        lbm.lbm_snapshot(self.h, 0, buf.data_ptr())
        return buf

    def restore(self, buf, t):
        lbm.lbm_restore(self.h, 0, buf.data_ptr())
        lbm.lbm_set_time(self.h, int(t))

    def step(self, n=1):
        lbm.lbm_step(self.h, n)

    @property
    def t(self):
        return lbm.lbm_time(self.h)

    def phi(self):
        return torch.as_tensor(self.sim.fields(0)[0], device=self.dev)

    def seed_phi(self, dphi):
        adj = self.new_state()
        dphi = dphi.to(device=self.dev, dtype=torch.float64).contiguous()
        lbm.lbm_adjoint_seed_phi(self.h, dphi.data_ptr(), adj.data_ptr())
        return adj

    def vjp_step(self, adj_in, grads=None, adj_out=None):
        """Adjoint of S_t from the adjoint of S_{t+1}.  Parameter derivatives
        accumulate on the device; with ``grads`` (numpy[6]) they are fetched."""
        if adj_out is None:
            adj_out = torch.empty((20,) + self.shape, dtype=self.dtype, device=self.dev)
        rc = lbm.lbm_adjoint_step(self.h, adj_in.data_ptr(), adj_out.data_ptr(), grads)
        if rc != lbm.LBM_OK:
            raise lbm.LbmError(rc, "lbm_adjoint_step", lbm.lib().lbm_last_error().decode())
        return adj_out

    def vjp_step_from(self, state, t, adj_in, adj_out=None):
        """Adjoint of S_t from the adjoint of S_{t+1}, for the snapshot
        ``state`` of S_t (the handle's own state is not used).  Parameter
        derivatives accumulate on the device."""
        if adj_out is None:
            adj_out = torch.empty((20,) + self.shape, dtype=self.dtype, device=self.dev)
        rc = lbm.lbm_adjoint_step_from(self.h, state.data_ptr(), int(t), adj_in.data_ptr(),
                                       adj_out.data_ptr(), None)
        if rc != lbm.LBM_OK:
            raise lbm.LbmError(rc, "lbm_adjoint_step_from", lbm.lib().lbm_last_error().decode())
        return adj_out

    def take_grads(self, grads):
        lbm.lbm_adjoint_take_param_grads(self.h, grads)

    def vjp_init(self, adj_state, grads):
        out = torch.zeros(self.shape, dtype=torch.float64, device=self.dev)
        lbm.lbm_adjoint_init(self.h, self.phi0.data_ptr(),
                             0 if self.u0 is None else self.u0.data_ptr(),
                             adj_state.data_ptr(), out.data_ptr(), grads)
        return out

    def close(self):
        self.sim.close()


def case_with(case, theta):
    c = dict(case)
    c["sigma"], c["tau_g"], c["lambda"] = float(theta[0]), float(theta[1]), float(theta[2])
    c["tau_f_l"] = c["tau_f_g"] = float(theta[3])
    if len(theta) > 4:
        c["u_top"], c["u_bot"] = float(theta[4]), float(theta[5])
    return c


def _stored_steps(nsteps, state_bytes, store_bytes, dev):
    """How many of the last steps keep their state in device memory."""
    if store_bytes is None:
        free, _ = torch.cuda.mem_get_info(dev)
        store_bytes = free // 4
    return int(max(0, min(nsteps, int(store_bytes) // state_bytes)))


class CoupledRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi0, theta, case, nsteps, ckpt_every, u0, store_bytes, tune, precision):
        th = theta.detach().cpu().numpy().astype(np.float64)
        asim = AdjointSim(case_with(case, th), phi0.detach().cpu().numpy(), u0, precision)
        if (nsteps >= 1000) if tune is None else bool(tune):
            asim.sim.autotune(1)  # the forward and the recomputation step with the fastest kernel
        state_bytes = lbm.lbm_snapshot_bytes(asim.h, 0)
        m = _stored_steps(nsteps, state_bytes, store_bytes, asim.dev)
        t_rec = nsteps - m  # states S_t, t in [t_rec, nsteps), stay on the device
        rec = torch.empty((m, asim.planes) + asim.shape, dtype=asim.dtype, device=asim.dev)
        ckpts = {0: asim.snapshot()} if t_rec > 0 else {}
        t = 0
        while t < t_rec:  # whole segments: the library replays CUDA graphs
            n = min(ckpt_every, t_rec - t)
            asim.step(n)
            t += n
            if t < t_rec:
                ckpts[t] = asim.snapshot()
        if m:  # snapshot and step, m times, in one library call
            lbm.lbm_record_steps(asim.h, m, rec.data_ptr(), rec[0].numel() * rec.element_size())
        phiT = asim.phi()
        ctx.asim, ctx.ckpts, ctx.rec, ctx.t_rec = asim, ckpts, rec, t_rec
        ctx.nsteps, ctx.k = nsteps, ckpt_every
        ctx.theta_dtype, ctx.theta_device = theta.dtype, theta.device
        ctx.ntheta = int(theta.numel())
        ctx.phi0_dtype, ctx.phi0_device = phi0.dtype, phi0.device
        return phiT

    @staticmethod
    def backward(ctx, grad_phiT):
        asim, nsteps, k, t_rec, rec = ctx.asim, ctx.nsteps, ctx.k, ctx.t_rec, ctx.rec
        grads = np.zeros(6)
        adj = asim.seed_phi(grad_phiT)
        spare = torch.empty_like(adj)
        # recorded states: no recomputation (one library call for the sweep)
        if nsteps > t_rec:
            lbm.lbm_adjoint_sweep(asim.h, rec.data_ptr(), rec[0].numel() * rec.element_size(),
                                  t_rec, nsteps - t_rec, adj.data_ptr(), spare.data_ptr())
        ctx.rec = rec = None
        # checkpointed segments below: recompute the states into one buffer,
        # then run the segment backwards
        if t_rec > 0:
            seg = torch.empty((min(k, t_rec),) + tuple(ctx.ckpts[0].shape), dtype=adj.dtype,
                              device=adj.device)
            stride = seg[0].numel() * seg.element_size()
        for t0 in reversed(sorted(ctx.ckpts)):
            t1 = min(t0 + k, t_rec)
            asim.restore(ctx.ckpts[t0], t0)
            lbm.lbm_record_steps(asim.h, t1 - t0, seg.data_ptr(), stride)
            lbm.lbm_adjoint_sweep(asim.h, seg.data_ptr(), stride, t0, t1 - t0, adj.data_ptr(),
                                  spare.data_ptr())
        if 0 in ctx.ckpts:
            asim.restore(ctx.ckpts[0], 0)
        dphi0 = asim.vjp_init(adj, None)
        asim.take_grads(grads)
        asim.close()
        gtheta = torch.as_tensor(grads[:ctx.ntheta], dtype=ctx.theta_dtype,
                                 device=ctx.theta_device)
        dphi0 = dphi0.to(device=ctx.phi0_device, dtype=ctx.phi0_dtype)
        return dphi0, gtheta, None, None, None, None, None, None, None


def coupled_run(phi0, theta, case, nsteps, ckpt_every=16, u0=None, store_bytes=None,
                tune=None, precision="f64"):
    """phi after nsteps coupled steps, differentiable in phi0 and theta.
    store_bytes bounds the device memory for recorded states (None: a
    quarter of the free memory; 0: checkpoints and recomputation only).
    tune: autotune the stepping kernel first (None: for runs of 1000 steps
    or more, where it pays for its trial steps).  precision: "f64", or "f32"
    for FP32 states, steps and adjoint arithmetic (phi returned in FP64)."""
    return CoupledRun.apply(phi0, theta, case, int(nsteps), int(ckpt_every), u0, store_bytes,
                            tune, precision)


def region_volume(phi, labels, region):
    """Phase volume sum(phi) over the nodes whose label is `region` (the
    droplet volumes of Fig. 3b): a linear objective of phi for the reverse
    mode.  phi: [ny][nx] tensor; labels: [ny][nx] integer array or tensor."""
    lab = torch.as_tensor(labels, device=phi.device)
    return (phi * (lab == region).to(phi.dtype)).sum()


def taylor_deformation(phi):
    """Taylor deformation D = (L - B)/(L + B) of a droplet from the second
    moments of phi about its centroid (L, B: semi-axes of the ellipse with
    those moments, proportional to the square roots of their eigenvalues).
    phi: [ny][nx] tensor; differentiable (torch autograd), for the shear-flow
    objective of the sheared-droplet set-up.  The droplet must not touch the
    periodic x-boundary."""
    ny, nx = phi.shape
    y = torch.arange(ny, dtype=phi.dtype, device=phi.device)[:, None]
    x = torch.arange(nx, dtype=phi.dtype, device=phi.device)[None, :]
    m = phi.sum()
    cx, cy = (phi * x).sum() / m, (phi * y).sum() / m
    dx, dy = x - cx, y - cy
    ixx, iyy, ixy = (phi * dx * dx).sum() / m, (phi * dy * dy).sum() / m, (phi * dx * dy).sum() / m
    # eigenvalues of [[ixx, ixy], [ixy, iyy]]
    half_tr, rad = 0.5 * (ixx + iyy), torch.sqrt(0.25 * (ixx - iyy) ** 2 + ixy * ixy)
    L, B = torch.sqrt(half_tr + rad), torch.sqrt(half_tr - rad)
    return (L - B) / (L + B)
