"""Gradient of the bottom-plate Nusselt number after K temperature steps with
respect to the initial temperature, as a ``torch.autograd.Function``.

The velocity history u^0 .. u^{K-1} comes from a Rayleigh-Benard run (the
Boussinesq BDF2/EXT2 step of Sec. 2.2 on the box of Sec. 4.4) and is frozen:
T^K is then an affine function of T^0 (Sec. 4.1, Eq. (2) with u given), and
the transposed steps of the library give its exact gradient. The history is
not stored: the run is checkpointed every ``every`` steps (device snapshots
of the full state) and each segment of velocities is regenerated from its
checkpoint when the forward or the reverse sweep reaches it, so at most
``every + 1`` velocity fields are held at a time.

Host logic only (the schedule of calls); every operation on the fields runs
in the library's kernels.
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import torch

from . import (RBC, TAdv, sem_bdf_ext_step, sem_rbc_fields, sem_rbc_load_state, sem_rbc_save_state,
               sem_tadv_adjoint_step, sem_tadv_nusselt, sem_tadv_nusselt_grad, sem_tadv_step)


class VelocityHistory:
    """The first K velocity levels of an RBC run, as checkpoints.

    Constructing it advances ``rbc`` by K steps, saving a snapshot before
    steps 0, every, 2 every, ...; afterwards ``rbc`` is left at step K.
    """

    def __init__(self, rbc: RBC, K: int, every: int = 5, stream=None):
        if K < 1 or every < 1:
            raise ValueError("need K >= 1 and every >= 1")
        self.rbc, self.K, self.every, self.stream = rbc, int(K), int(every), stream
        self.snaps = []
        self.stats: List[dict] = []
        self.n_replayed = 0
        for n in range(self.K):
            if n % self.every == 0:
                self.snaps.append(sem_rbc_save_state(rbc, stream=stream))
            self.stats.append(sem_bdf_ext_step(rbc, stream=stream))
        self.final = sem_rbc_save_state(rbc, stream=stream)

    @property
    def n_segments(self) -> int:
        return len(self.snaps)

    def bounds(self, s: int) -> Tuple[int, int]:
        return s * self.every, min((s + 1) * self.every, self.K)

    def segment(self, s: int) -> Dict[int, list]:
        """Velocities u^n for n in [n0 - 1, n1) of segment s (n0 - 1 only when
        n0 > 0), regenerated from the segment's checkpoint."""
        n0, n1 = self.bounds(s)
        sem_rbc_load_state(self.rbc, self.snaps[s], stream=self.stream)
        f = sem_rbc_fields(self.rbc)
        vel = {n0: [f["u"], f["v"], f["w"]]}
        if n0 > 0:
            vel[n0 - 1] = [f["u_prev"], f["v_prev"], f["w_prev"]]
        for n in range(n0 + 1, n1):
            sem_bdf_ext_step(self.rbc, stream=self.stream)
            self.n_replayed += 1
            f = sem_rbc_fields(self.rbc)
            vel[n] = [f["u"], f["v"], f["w"]]
        return vel

    def restore(self):
        sem_rbc_load_state(self.rbc, self.final, stream=self.stream)

    def transport(self, tadv: TAdv, T0):
        """T^K from T^0 with the frozen velocities (forward sweep)."""
        m = tadv.mesh
        Tn, Tnm1, NTnm1 = T0.contiguous(), None, None
        for s in range(self.n_segments):
            vel = self.segment(s)
            n0, n1 = self.bounds(s)
            for n in range(n0, n1):
                Tnp1 = torch.empty_like(Tn)
                NTn = torch.empty(m.n_local, dtype=torch.float64, device=Tn.device)
                sem_tadv_step(tadv, n, vel[n], Tn, Tnm1, NTnm1, Tnp1, NTn, stream=self.stream)
                Tnm1, Tn, NTnm1 = Tn, Tnp1, NTn
        self.restore()
        return Tn

    def adjoint(self, tadv: TAdv, gK):
        """dJ/dT^0 on the free nodes for J = gK . T^K (reverse sweep)."""
        g_np1 = gK.contiguous().clone()
        g_n = torch.zeros_like(g_np1)
        g_nm1 = torch.zeros_like(g_np1)
        for s in range(self.n_segments - 1, -1, -1):
            vel = self.segment(s)
            n0, n1 = self.bounds(s)
            for n in range(n1 - 1, n0 - 1, -1):
                sem_tadv_adjoint_step(tadv, n, vel[n], vel.get(n - 1), g_np1, g_n, g_nm1 if n > 0 else None,
                                      stream=self.stream)
                if n > 0:  # g^n is complete; g^{n-1} holds step n's share
                    g_np1, g_n, g_nm1 = g_n, g_nm1, g_np1
                    g_nm1.zero_()
        self.restore()
        return g_n


class NusseltOfT0(torch.autograd.Function):
    """Nu_b(T^K) as a function of T^0 (U-vector, float64, on the GPU)."""

    @staticmethod
    def forward(ctx, T0, hist: VelocityHistory, tadv: TAdv):
        TK = hist.transport(tadv, T0)
        ctx.hist, ctx.tadv = hist, tadv
        return torch.tensor(sem_tadv_nusselt(tadv, TK, stream=hist.stream), dtype=torch.float64, device=T0.device)

    @staticmethod
    def backward(ctx, gout):
        hist, tadv = ctx.hist, ctx.tadv
        gK = torch.empty(tadv.mesh.n_unique, dtype=torch.float64, device=gout.device)
        sem_tadv_nusselt_grad(tadv, gK, scale=float(gout), stream=hist.stream)
        return hist.adjoint(tadv, gK), None, None


def nusselt_after(T0, hist: VelocityHistory, tadv: TAdv):
    """Differentiable Nu_b(T^K) of the initial temperature T0."""
    return NusseltOfT0.apply(T0, hist, tadv)
