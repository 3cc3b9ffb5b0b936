"""torch-facing wrappers of the bpimd library.

``ExchangeEnergy`` owns one C-ABI context (``bpimd_create``) bound to the
current CUDA stream and evaluates V^{[1,N]} and the bead forces of Algorithm 1
on device tensors.  ``exchange_potential`` is the autograd form: its forward
returns V^{[1,N]}; its backward multiplies the incoming gradient by -F, where F
is the force the same kernel pass produced (the connection-probability force
expression of Lemma expected-force is exactly -grad V), so no O(N^2) tensor is
saved for backward.
"""
import torch

from . import bpimd as _c


class ExchangeEnergy:
    """Exchange potential and forces for one system of N particles, P beads."""

    def __init__(self, N, P, m, omega_P, beta, precision="fp64", device="cuda", stream=None, box=0.0,
                 recompute=False):
        """recompute=True: no O(N^2) storage at any N (automatic above
        BPIMD_STORE_MAX_N): the pair factors are recomputed where used."""
        if not torch.cuda.is_available():
            raise RuntimeError("bpimd needs a CUDA device; there is no CPU fallback")
        prec = _c.PRECISIONS[precision]
        self.N, self.P = int(N), int(P)
        self.m, self.omega_P, self.beta = float(m), float(omega_P), float(beta)
        self.precision = precision
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise ValueError("bpimd runs on CUDA devices only")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.cfg = _c.make_config(self.N, self.P, self.m, self.omega_P, self.beta, prec, box_L=float(box),
                                      flags=_c.BPIMD_FLAG_RECOMPUTE if recompute else 0)
            self.ctx = _c.bpimd_create(self.cfg, self.stream)
            self._V = torch.empty((), dtype=torch.float64, device=self.device)

    def close(self):
        if getattr(self, "ctx", None):
            _c.bpimd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, pos):
        if pos.dtype != torch.float64 or pos.device != self.device or tuple(pos.shape) != (self.N, self.P, 3):
            raise ValueError(f"positions must be float64 [{self.N}][{self.P}][3] on {self.device}")
        return pos.contiguous()

    def forces(self, pos, out=None, V_out=None):
        """Enqueue one evaluation; returns (V_B 0-d tensor, forces)."""
        pos = self._check(pos)
        F = out if out is not None else torch.empty_like(pos)
        V = V_out if V_out is not None else torch.empty((), dtype=torch.float64, device=self.device)
        _c.bpimd_exchange_energy_forces(self.ctx, pos, V, F)
        return V, F

    __call__ = forces

    def forces_host(self, pos_host, F_host=None):
        """Host-buffer entry point (copies in and out, synchronises)."""
        import numpy as np
        F_host = F_host if F_host is not None else torch.empty_like(pos_host)
        V = np.zeros(1)
        _c.bpimd_exchange_energy_forces_host(self.ctx, pos_host, V, F_host)
        return float(V[0]), F_host

    def potentials(self):
        """(V^{[1,v]} for v=0..N, V^{[u,N]} for u=1..N+1, E_int) of the last evaluation."""
        import numpy as np
        Vf, Vb, Ei = np.empty(self.N + 1), np.empty(self.N + 1), np.empty(self.N)
        _c.bpimd_get_potentials(self.ctx, Vf, Vb, Ei)
        return Vf, Vb, Ei

    def connection_probabilities(self):
        """Dense N x N matrix Pr[l -> l'] of the last evaluation (device tensor)."""
        M = torch.empty((self.N, self.N), dtype=torch.float64, device=self.device)
        _c.bpimd_connection_probabilities(self.ctx, M)
        return M

    def sync(self):
        _c.bpimd_sync(self.ctx)


class _ExchangeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, engine):
        V, F = engine.forces(pos)
        ctx.save_for_backward(F)
        return V

    @staticmethod
    def backward(ctx, gV):
        (F,) = ctx.saved_tensors
        return -gV * F, None


def exchange_potential(pos, engine):
    """V^{[1,N]}(pos) as a differentiable scalar; d/dpos is -F from the force kernel."""
    return _ExchangeFn.apply(pos, engine)


class RingPolymerMD:
    """BAOAB Langevin molecular dynamics of N bosonic ring polymers (bpimd_step).

    Samples exp(-beta (V^{[1,N]} + U-bar)) with the exchange force of Algorithm 1
    plus a harmonic trap (omega0) and an optional Gaussian repulsion
    g exp(-r^2/(2 s^2)) or Lennard-Jones pair potential (eps, sigma, cutoff;
    truncated and shifted) between beads of equal index; box > 0 makes the
    system periodic (minimum-image springs and pairs; Lennard-Jones by cell
    lists when the box holds at least 3 cutoffs per side).  ``step`` advances the
    caller's position and velocity tensors in place; with a non-default stream
    the step runs as a replayed CUDA graph.
    """

    def __init__(self, N, P, m, omega_P, beta, dt, gamma=1.0, omega0=0.0, gaussian=None, kT=0.0,
                 seed=0, precision="fp64", device="cuda", stream=None, lennard_jones=None, box=0.0,
                 recompute=False):
        if not torch.cuda.is_available():
            raise RuntimeError("bpimd needs a CUDA device; there is no CPU fallback")
        prec = _c.PRECISIONS[precision]
        self.N, self.P = int(N), int(P)
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        md = dict(dt=float(dt), gamma=float(gamma), kT_bead=float(kT), omega0=float(omega0), seed=int(seed))
        if gaussian is not None:
            md.update(pair_type=_c.BPIMD_PAIR_GAUSSIAN, pair_a=float(gaussian[0]), pair_b=float(gaussian[1]))
        if lennard_jones is not None:  # (eps, sigma, cutoff)
            md.update(pair_type=_c.BPIMD_PAIR_LJ, pair_a=float(lennard_jones[0]), pair_b=float(lennard_jones[1]),
                      pair_rc=float(lennard_jones[2]))
        md["box_L"] = float(box)
        md["flags"] = _c.BPIMD_FLAG_RECOMPUTE if recompute else 0
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.cfg = _c.make_config(self.N, self.P, float(m), float(omega_P), float(beta), prec, **md)
            self.ctx = _c.bpimd_create(self.cfg, self.stream)
            self.energies = torch.zeros(4, dtype=torch.float64, device=self.device)

    def close(self):
        if getattr(self, "ctx", None):
            _c.bpimd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, pos, vel, nsteps=1, energies=True):
        """Advance (pos, vel) by nsteps; returns the device tensor
        [V_B, U-bar, kinetic, primitive estimator] after the last step, or None."""
        for t in (pos, vel):
            if t.dtype != torch.float64 or t.device != self.device or tuple(t.shape) != (self.N, self.P, 3) \
                    or not t.is_contiguous():
                raise ValueError(f"positions/velocities must be contiguous float64 [{self.N}][{self.P}][3]")
        _c.bpimd_step(self.ctx, pos, vel, nsteps, self.energies if energies else None)
        return self.energies if energies else None


class BatchedExchangeEnergy:
    """V^{[1,N_r]} and forces of R independent replicas in one evaluation.

    Replica r has N[r] particles, P[r] beads, omega_P[r], beta[r] (shared mass
    and precision).  Positions and forces are packed: replica r is the
    [N_r][P_r][3] block at element offset ``offsets[r]`` of one flat float64
    tensor (``pack``/``unpack`` convert from/to lists of tensors).  Three kernel
    launches per evaluation regardless of R (plus one per replica above 4096
    particles); ``step`` runs BAOAB molecular dynamics of every replica.
    """

    def __init__(self, N, P, m, omega_P, beta, precision="fp64", device="cuda", stream=None, md=None):
        """md: optional molecular-dynamics parameters for ``step`` (dt, gamma,
        omega0, gaussian=(g, s), kT, seed), shared by all replicas."""
        if not torch.cuda.is_available():
            raise RuntimeError("bpimd needs a CUDA device; there is no CPU fallback")
        prec = _c.PRECISIONS[precision]
        self.N = [int(n) for n in N]
        self.P = [int(p) for p in P]
        self.R = len(self.N)
        self.precision = precision
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            kw = {}
            if md:
                kw = dict(dt=float(md.get("dt", 0.0)), gamma=float(md.get("gamma", 1.0)),
                          kT_bead=float(md.get("kT", 0.0)), omega0=float(md.get("omega0", 0.0)),
                          seed=int(md.get("seed", 0)))
                if md.get("gaussian") is not None:
                    kw.update(pair_type=_c.BPIMD_PAIR_GAUSSIAN, pair_a=float(md["gaussian"][0]),
                              pair_b=float(md["gaussian"][1]))
            cfg = _c.make_config(0, 0, float(m), 1.0, 1.0, prec, **kw)
            self.ctx = _c.bpimd_create_batched(cfg, self.N, self.P, omega_P, beta, self.stream)
            self.energies = torch.zeros((self.R, 4), dtype=torch.float64, device=self.device)
        _, self.elements, self.offsets = _c.bpimd_batch_info(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            _c.bpimd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pack(self, tensors):
        """List of [N_r][P_r][3] tensors -> one packed float64 tensor on the device."""
        return torch.cat([t.reshape(-1) for t in tensors]).to(device=self.device, dtype=torch.float64).contiguous()

    def unpack(self, packed):
        """Packed tensor -> list of [N_r][P_r][3] views."""
        out = []
        for r in range(self.R):
            o = int(self.offsets[r])
            out.append(packed[o:o + 3 * self.N[r] * self.P[r]].view(self.N[r], self.P[r], 3))
        return out

    def forces(self, packed, out=None, V_out=None):
        """Enqueue one evaluation; returns (V_B [R] tensor, packed forces)."""
        if packed.dtype != torch.float64 or packed.device != self.device or packed.numel() != self.elements \
                or not packed.is_contiguous():
            raise ValueError(f"positions must be a contiguous packed float64 tensor of {self.elements} elements")
        F = out if out is not None else torch.empty_like(packed)
        V = V_out if V_out is not None else torch.empty(self.R, dtype=torch.float64, device=self.device)
        _c.bpimd_exchange_energy_forces_batched(self.ctx, packed, V, F)
        return V, F

    __call__ = forces

    def set_tuning(self, pair_blocks_per_sm, prob_blocks_per_sm):
        _c.bpimd_batch_set_tuning(self.ctx, pair_blocks_per_sm, prob_blocks_per_sm)

    def set_pair_tile(self, lanes_per_particle):
        """Pair tile of ``step``'s trap and pair forces: 2, 4 or 8 lanes per particle."""
        _c.bpimd_batch_set_pair_tile(self.ctx, lanes_per_particle)

    def step(self, pos, vel, nsteps=1, energies=True):
        """Advance every replica by nsteps BAOAB steps (packed pos, vel in
        place); returns the device tensor [R][4] of (V_B, U-bar, kinetic,
        primitive estimator) per replica after the last step, or None."""
        for t in (pos, vel):
            if t.dtype != torch.float64 or t.device != self.device or t.numel() != self.elements \
                    or not t.is_contiguous():
                raise ValueError(f"positions/velocities must be contiguous packed float64 of {self.elements}")
        _c.bpimd_step(self.ctx, pos, vel, nsteps, self.energies if energies else None)
        return self.energies if energies else None

    def sync(self):
        _c.bpimd_sync(self.ctx)
