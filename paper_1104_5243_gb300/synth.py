"""Seeded synthetic inputs shaped like an interventional C-arm acquisition.

This module only *generates inputs*: scan parameters, projection angles,
random projection stacks and random ellipsoid phantom parameters.  It holds
none of the backprojection arithmetic; the CUDA library and the CPU oracle
both take their inputs from here and compute everything else on their own.

Workload shapes follow the paper's RabbitCT case (Sect. 3.1): a 256 mm cube
volume of L^3 voxels and projections of ISX x ISY pixels.  The RabbitCT rabbit
data set is not available, so seeded synthetic stacks stand in for it:

* C-arm circular short scan over 200 degrees, source-isocenter 785 mm,
  source-detector 1200 mm, uniform angles beta_i = beta_0 + i * 200deg/(N-1),
  rotation about z, principal point at the detector centre.
* timing stack: uniform [0, 1) float32 projections (PCG64 seed 20110426);
* phantoms: random ellipsoids with densities U[0.1, 1] (scaled by 0.02/mm so
  line integrals are water-like), semi-axes U[8, 64] mm, uniform random
  orientation, centres inside 0.8 x the field-of-view cylinder (clipped to
  the 256 mm cube).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SID_MM = 785.0          # source to isocenter
SDD_MM = 1200.0         # source to detector
SCAN_DEG = 200.0        # short-scan arc
VOLUME_MM = 256.0       # edge of the reconstructed cube (Sect. 3.1, Fig. 1)
TIMING_SEED = 20110426  # uniform timing stack
DENSITY_SCALE = 0.02    # mm^-1 per unit phantom density


@dataclasses.dataclass(frozen=True)
class Scan:
    """One C-arm acquisition: detector size/pitch and projection angles."""
    n: int              # number of projections
    isx: int            # detector columns (u)
    isy: int            # detector rows (v)
    pitch: float        # square pixel pitch on the detector, mm
    sid: float = SID_MM
    sdd: float = SDD_MM
    scan_deg: float = SCAN_DEG
    beta0_deg: float = 0.0

    @property
    def betas(self) -> np.ndarray:
        """Projection angles in radians (float64)."""
        if self.n == 1:
            return np.array([math.radians(self.beta0_deg)])
        step = self.scan_deg / (self.n - 1)
        return np.radians(self.beta0_deg + step * np.arange(self.n, dtype=np.float64))

    @property
    def cu(self) -> float:
        return (self.isx - 1) / 2.0

    @property
    def cv(self) -> float:
        return (self.isy - 1) / 2.0


@dataclasses.dataclass(frozen=True)
class Volume:
    """L^3 voxel grid of the 256 mm cube centred at the isocenter."""
    L: int

    @property
    def R(self) -> float:
        """Voxel size in mm."""
        return VOLUME_MM / self.L

    @property
    def O(self) -> tuple:
        """World position (mm) of the centre of voxel (0, 0, 0)."""
        o = -self.R * (self.L - 1) / 2.0
        return (o, o, o)


# --- workloads (detector sizes and pitches keep the 384 x 295.7 mm panel) ---
SCANS = {
    "tiny": Scan(n=36, isx=160, isy=120, pitch=7.68),
    "full": Scan(n=496, isx=1248, isy=960, pitch=0.308),
    "half": Scan(n=248, isx=624, isy=480, pitch=0.616),
    "grad": Scan(n=12, isx=64, isy=48, pitch=6.006),
    "train": Scan(n=120, isx=312, isy=240, pitch=1.232),
}


def uniform_stack(n: int, isy: int, isx: int, seed: int = TIMING_SEED) -> np.ndarray:
    """Uniform [0, 1) float32 projection stack, shape (n, isy, isx)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random((n, isy, isx), dtype=np.float32)


def uniform_volume(L: int, seed: int) -> np.ndarray:
    """Uniform [0, 1) float32 volume, shape (L, L, L) indexed [z, y, x]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random((L, L, L), dtype=np.float32)


def field_of_view(scan: Scan) -> tuple:
    """(radius, half height) in mm of the cylinder seen by every projection."""
    half_w = scan.isx * scan.pitch / 2.0
    half_h = scan.isy * scan.pitch / 2.0
    radius = scan.sid * math.sin(math.atan(half_w / scan.sdd))
    return radius, half_h * scan.sid / scan.sdd


def ellipsoids(count: int, seed: int, scan: Scan) -> np.ndarray:
    """Random ellipsoid phantom, float64 array (count, 16).

    Row layout: centre (3), semi-axes (3), rotation matrix (9, row-major; its
    columns are the ellipsoid axes in world coordinates), density (1, mm^-1).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    radius, half_h = field_of_view(scan)
    # centres inside the field of view and inside the reconstructed cube
    radius = min(radius, VOLUME_MM / 2)
    half_h = min(half_h, VOLUME_MM / 2)
    out = np.zeros((count, 16), dtype=np.float64)
    for e in range(count):
        rr = 0.8 * radius * math.sqrt(rng.random())
        phi = 2.0 * math.pi * rng.random()
        cz = 0.8 * half_h * (2.0 * rng.random() - 1.0)
        axes = rng.uniform(8.0, 64.0, size=3)
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        a, b, c, d = q
        rot = np.array([
            [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
            [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
            [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
        ])
        out[e, 0:3] = (rr * math.cos(phi), rr * math.sin(phi), cz)
        out[e, 3:6] = axes
        out[e, 6:15] = rot.reshape(-1)
        out[e, 15] = DENSITY_SCALE * rng.uniform(0.1, 1.0)
    return out


def sphere(centre, radius: float, density: float) -> np.ndarray:
    """A single axis-aligned sphere in the ellipsoid row layout, shape (1, 16)."""
    row = np.zeros((1, 16), dtype=np.float64)
    row[0, 0:3] = centre
    row[0, 3:6] = radius
    row[0, 6:15] = np.eye(3).reshape(-1)
    row[0, 15] = density
    return row


def poisson_counts(line_integrals: np.ndarray, photons: float, seed: int) -> np.ndarray:
    """Poisson photon counts I ~ Poisson(I0 * exp(-l)) for each ray (float64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.poisson(photons * np.exp(-np.asarray(line_integrals, dtype=np.float64))).astype(np.float64)


def noisy_line_integrals(lines, photons: float, seed: int):
    """Measured line integrals -log(max(I, 1) / I0) with photon counts
    I ~ Poisson(I0 exp(-l)), drawn by torch on the tensor's device with a
    generator seeded by `seed` (float32 tensor in, float32 tensor out)."""
    import torch
    g = torch.Generator(device=lines.device)
    g.manual_seed(int(seed))
    counts = torch.poisson(photons * torch.exp(-lines.double()), generator=g)
    return (-torch.log(torch.clamp(counts, min=1.0) / photons)).float()
