"""Differentiable backprojection and the learned per-row FDK filter.

* ``BackprojectFn``: vol = B(p) with B the voxel-driven backprojection of
  Sect. 3.1 (Listing 1); its backward is the hand-written adjoint kernel
  (bp_adjoint, a voxel-driven forward projection with atomic scatter), the
  exact transpose of B.
* ``RowFilterFn``: the short per-row convolution with T taps; backward runs
  the row-filter gradient kernel (input gradient and a deterministic
  two-pass tap reduction).
* ``LearnedRowFilter``: T learned taps (default 64) that replace the central
  T taps of the Ram-Lak ramp in the 2-D FDK pre-processing (Sect. 1.1 names
  the step; the cosine and Parker weights stay fixed).  The ramp's tails
  beyond +-T/2 pixels stay analytic: they carry the |omega| response at low
  frequencies, which no short filter can represent, and no noise trade-off.
  Initialised to the Ram-Lak kernel (so training starts from the plain
  FDK), trained on phantoms this package projects itself, judged against the
  phantom and against the plain ramp-filter FDK, which stays available as
  the fallback (``ramp_fdk``).

Every computation on the data path runs in libbp1104.so; PyTorch provides the
tensors, the autograd tape, the loss and the optimiser.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

from . import api, synth


class BackprojectFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, proj: torch.Tensor, bp: api.Backprojector, A: np.ndarray):
        bp.reset()
        bp.add_projections(proj, A)
        vol = bp.finalize()
        ctx.bp, ctx.A = bp, A
        return vol

    @staticmethod
    def backward(ctx, gvol: torch.Tensor):
        if not ctx.needs_input_grad[0]:
            return None, None, None
        return ctx.bp.adjoint(gvol.contiguous(), ctx.A), None, None


def backproject(proj: torch.Tensor, bp: api.Backprojector, A) -> torch.Tensor:
    """Differentiable backprojection of proj (n, isy, isx) into bp's volume."""
    return BackprojectFn.apply(proj, bp, A)


class RowFilterFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, h: torch.Tensor):
        x, h = x.contiguous(), h.contiguous()
        ctx.save_for_backward(x, h)
        return api.row_filter_fwd(x, h)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        x, h = ctx.saved_tensors
        gin, gh = api.row_filter_bwd(x, h, g.contiguous(), need_x=ctx.needs_input_grad[0],
                                     need_h=ctx.needs_input_grad[1])
        return gin, gh


def row_filter(x: torch.Tensor, h: torch.Tensor) -> torch.Tensor:
    return RowFilterFn.apply(x, h)


def ramlak_taps(T: int, tau: float, scale: float = 1.0) -> np.ndarray:
    """Ram-Lak kernel (h(0) = 1/(4 tau^2), h(odd m) = -1/(m^2 pi^2 tau^2))
    times tau, truncated to T taps in the row filter's layout: tap t weighs
    the pixel at offset m = t - T/2."""
    m = np.arange(T) - T // 2
    h = np.where(m == 0, 1.0 / (4 * tau * tau),
                 np.where(m % 2 != 0, -1.0 / (np.maximum(m * m, 1) * math.pi ** 2 * tau * tau), 0.0))
    return (scale * tau * h).astype(np.float32)


class LearnedRowFilter(torch.nn.Module):
    """The ramp filter with its central T taps learned:
    q = ramp(x) + (taps - ramlak_central) * x along every detector row, where
    ramp is the full-length Ram-Lak filter at isocenter pitch tau.

    The learned change of the taps is symmetric and parameterised by its
    frequency response: delta(m) = sum_k coef[k] cos(2 pi k m / T) for the
    T/2 + 1 frequencies k (the "response" form of the learned filter).  Each
    parameter then moves one frequency band, which keeps the optimisation
    well conditioned: in the tap basis the low-frequency (DC) direction,
    to which the reconstruction error is by far most sensitive, dominates
    every tap's gradient.

    response="cosine" (default) learns the T/2 + 1 coefficients directly;
    response="mlp" makes them the output of a small multilayer perceptron of
    the normalised frequency k / (T/2) (1 -> hidden -> hidden -> 1, tanh),
    a smooth response with fewer degrees of freedom per band.  Its last layer
    starts at zero, so either form starts from the plain ramp."""

    def __init__(self, T: int = 64, tau: float = 1.0, response: str = "cosine", hidden: int = 16):
        super().__init__()
        if response not in ("cosine", "mlp"):
            raise ValueError(f"response must be 'cosine' or 'mlp', got {response!r}")
        self.tau = float(tau)
        self.response = response
        central = torch.from_numpy(ramlak_taps(T, tau))
        m = torch.arange(T, dtype=torch.float64) - T // 2
        k = torch.arange(T // 2 + 1, dtype=torch.float64)
        basis = torch.cos(2.0 * math.pi * m[:, None] * k[None, :] / T).float()
        self.register_buffer("ramlak_central", central)
        self.register_buffer("basis", basis)
        if response == "cosine":
            self.coef = torch.nn.Parameter(torch.zeros(T // 2 + 1))
        else:
            self.register_buffer("freq", (k / (T // 2)).float()[:, None])
            self.mlp = torch.nn.Sequential(torch.nn.Linear(1, hidden), torch.nn.Tanh(),
                                           torch.nn.Linear(hidden, hidden), torch.nn.Tanh(),
                                           torch.nn.Linear(hidden, 1))
            torch.nn.init.zeros_(self.mlp[-1].weight)
            torch.nn.init.zeros_(self.mlp[-1].bias)
            # output scale 1 / hidden: an Adam step of the last layer (hidden
            # weights) then moves a coefficient about as far as one step of
            # the cosine form, so both train at the same learning rate
            self.out_scale = 1.0 / hidden

    def coefficients(self) -> torch.Tensor:
        """The T/2 + 1 cosine coefficients of the learned change."""
        if self.response == "cosine":
            return self.coef
        return self.mlp(self.freq).squeeze(-1) * self.out_scale

    @property
    def delta(self) -> torch.Tensor:
        return self.basis @ self.coefficients()

    def delta_at_pitch(self, factor: int) -> torch.Tensor:
        """The learned change resampled to a detector `factor` times finer:
        the same cosine series evaluated at m / factor and scaled by
        1 / factor (the row filter approximates a convolution integral, so
        taps scale with the pixel pitch); factor * T taps."""
        T = self.basis.shape[0]
        dev = self.basis.device
        m = (torch.arange(T * factor, dtype=torch.float64, device=dev) - T * factor // 2) / factor
        k = torch.arange(T // 2 + 1, dtype=torch.float64, device=dev)
        basis = torch.cos(2.0 * math.pi * m[:, None] * k[None, :] / T)
        return (basis @ self.coefficients().detach().double() / factor).float()

    @property
    def taps(self) -> torch.Tensor:
        """The learned central taps (Ram-Lak central taps + learned change)."""
        return self.ramlak_central + self.delta

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        with torch.no_grad():
            base = api.ramp_filter(x, self.tau)
        return base + row_filter(x, self.delta.contiguous())


# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    """Training workload: 128^3 volume, 120 projections of 312 x 240."""
    scan: synth.Scan = dataclasses.field(default_factory=lambda: synth.SCANS["train"])
    L: int = 128
    ellipsoids: int = 10
    photons: float = 1e4

    @property
    def volume(self):
        return synth.Volume(self.L)


class PhantomData:
    """Noisy pre-weighted projections and voxelised targets of seeded
    phantoms, generated on the GPU by this package's kernels."""

    def __init__(self, wl: Workload, A: np.ndarray):
        self.wl, self.A = wl, A

    def sample(self, seed: int):
        wl, scan, vol = self.wl, self.wl.scan, self.wl.volume
        ell = synth.ellipsoids(wl.ellipsoids, seed=seed, scan=scan)
        lines = api.ellipsoid_project(self.A, scan.isx, scan.isy, ell)
        noisy = synth.noisy_line_integrals(lines, wl.photons, seed)
        pre = api.fdk_preweight(scan, noisy, parker=True, scale=api.fdk_scale(scan))
        target = api.ellipsoid_voxelize(vol.L, vol.R, vol.O, ell)
        return pre, target


def ramp_fdk(pre: torch.Tensor, scan, bp: api.Backprojector, A) -> torch.Tensor:
    """The plain FDK: Ram-Lak ramp filter of the pre-weighted projections,
    then backprojection (the fallback and the yardstick)."""
    bp.reset()
    bp.add_projections(api.ramp_filter(pre, api.iso_pitch(scan)), A)
    return bp.finalize()


def train(steps: int = 200, batch: int = 8, T: int = 64, lr: float = 1e-4, seed0: int = 1000,
          wl: Workload | None = None, log=None, response: str = "cosine"):
    """Train the taps through the GPU forward and backward kernels on batches
    of seeded phantoms (seeds seed0 + k); response selects the filter's
    parameterisation (LearnedRowFilter).  Returns (module, losses)."""
    wl = wl or Workload()
    scan, vol = wl.scan, wl.volume
    A = api.carm_matrices(scan)
    data = PhantomData(wl, A)
    filt = LearnedRowFilter(T, tau=api.iso_pitch(scan), response=response).cuda()
    opt = torch.optim.Adam(filt.parameters(), lr=lr)
    bp = api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy)
    pool = [data.sample(seed0 + k) for k in range(batch * 4)]
    losses = []
    for it in range(steps):
        opt.zero_grad(set_to_none=True)
        total = 0.0
        for b in range(batch):
            pre, target = pool[(it * batch + b) % len(pool)]
            volume = backproject(filt(pre), bp, A)
            loss = torch.mean((volume - target) ** 2) / batch
            loss.backward()
            total += float(loss.detach())
        opt.step()
        losses.append(total)
        if log is not None and (it % 25 == 0 or it == steps - 1):
            log(f"step {it:4d} loss {total:.4e}")
    bp.close()
    return filt, losses


@torch.no_grad()
def full_size_inference(filt: LearnedRowFilter, seeds, L: int = 512, ellipsoids: int = 10,
                        train: Workload | None = None) -> dict:
    """Apply a filter trained on the 312 x 240 detector to the full
    1248 x 960 x 496 scan and a 512^3 volume, judged against the phantom and
    against the plain ramp FDK.  The detector pitch is 4x finer, so the
    learned change is resampled to 4x the taps, and the photon count per
    pixel is scaled by the pixel area (the same dose per mm^2)."""
    train = train or Workload()
    full = synth.SCANS["full"]
    factor = int(round(train.scan.pitch / full.pitch))
    photons = train.photons * (full.pitch / train.scan.pitch) ** 2
    vol = synth.Volume(L)
    A = api.carm_matrices(full)
    bp = api.Backprojector(vol.L, vol.R, vol.O, full.isx, full.isy)
    delta = filt.delta_at_pitch(factor).contiguous()
    tau = api.iso_pitch(full)
    mse_l, mse_r = [], []
    for s in seeds:
        ell = synth.ellipsoids(ellipsoids, seed=s, scan=train.scan)
        lines = api.ellipsoid_project(A, full.isx, full.isy, ell)
        noisy = synth.noisy_line_integrals(lines, photons, s)
        del lines
        pre = api.fdk_preweight(full, noisy, parker=True, scale=api.fdk_scale(full))
        del noisy
        target = api.ellipsoid_voxelize(vol.L, vol.R, vol.O, ell)
        ramp = api.ramp_filter(pre, tau)
        bp.reset()
        bp.add_projections(ramp, A)
        v_r = bp.finalize()
        mse_r.append(float(torch.mean((v_r - target) ** 2)))
        del v_r
        ramp += api.row_filter_fwd(pre, delta)
        bp.reset()
        bp.add_projections(ramp, A)
        v_l = bp.finalize()
        mse_l.append(float(torch.mean((v_l - target) ** 2)))
        del v_l, ramp, pre, target
    bp.close()
    return {"mse_learned": float(np.mean(mse_l)), "mse_ramp": float(np.mean(mse_r)),
            "per_seed_learned": mse_l, "per_seed_ramp": mse_r, "taps": int(delta.numel()),
            "photons_per_pixel": photons}


@torch.no_grad()
def evaluate(filt: LearnedRowFilter, seeds, wl: Workload | None = None) -> dict:
    """Mean squared error against the phantom of the learned-filter FDK and
    of the plain ramp FDK on the given (held-out) seeds."""
    wl = wl or Workload()
    scan, vol = wl.scan, wl.volume
    A = api.carm_matrices(scan)
    data = PhantomData(wl, A)
    bp = api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy)
    mse_l, mse_r = [], []
    for s in seeds:
        pre, target = data.sample(s)
        bp.reset()
        bp.add_projections(filt(pre), A)
        v_l = bp.finalize()
        v_r = ramp_fdk(pre, scan, bp, A)
        mse_l.append(float(torch.mean((v_l - target) ** 2)))
        mse_r.append(float(torch.mean((v_r - target) ** 2)))
    bp.close()
    return {"mse_learned": float(np.mean(mse_l)), "mse_ramp": float(np.mean(mse_r)),
            "per_seed_learned": mse_l, "per_seed_ramp": mse_r}
