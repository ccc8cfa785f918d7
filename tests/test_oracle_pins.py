"""Pins for the FP64 CPU oracle: each checks it against something other than
itself -- an independent geometric construction, exact rational arithmetic,
closed forms, invariants of the linear map, or a library routine -- so that a
dropped term, a wrong sign, a transposed operand or an off-by-one index in the
oracle fails at least one of them.  CPU only.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1104_5243_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# An independent construction of the C-arm projection: ray from the source
# through the voxel, intersected with the detector plane (no matrix at all).
def geometric_projection(scan, beta, X):
    c, s = math.cos(beta), math.sin(beta)
    S = np.array([scan.sid * c, scan.sid * s, 0.0])
    d = np.array([-c, -s, 0.0])              # central ray, source -> isocenter
    eu = np.array([-s, c, 0.0])
    ev = np.array([0.0, 0.0, 1.0])
    X = np.asarray(X, dtype=np.float64)
    depth = float((X - S) @ d)
    P = S + (X - S) * (scan.sdd / depth)     # hit point on the detector plane
    Dc = S + scan.sdd * d                    # detector centre
    u = float((P - Dc) @ eu) / scan.pitch + scan.cu
    v = float((P - Dc) @ ev) / scan.pitch + scan.cv
    return u, v, depth / scan.sid


def listing_sample(img, u, v):
    """The listing's Part 2 + Part 3 for one voxel, with explicit corner tests."""
    isy, isx = img.shape
    iu, iv = math.floor(u), math.floor(v)
    sx, sy = u - iu, v - iv
    tl = tr = bl = br = 0.0
    if 0 <= iv < isy:
        if 0 <= iu < isx:
            tl = float(img[iv, iu])
        if -1 <= iu < isx - 1:
            tr = float(img[iv, iu + 1])
    if -1 <= iv < isy - 1:
        if 0 <= iu < isx:
            bl = float(img[iv + 1, iu])
        if -1 <= iu < isx - 1:
            br = float(img[iv + 1, iu + 1])
    vall = sy * bl + (1 - sy) * tl
    valr = sy * br + (1 - sy) * tr
    return sx * valr + (1 - sx) * vall


SMALL = synth.Scan(n=6, isx=20, isy=16, pitch=19.0)


def test_matrices_match_ray_plane_intersection():
    scan = synth.SCANS["full"]
    A = oracle.carm_matrices(scan)
    rng = np.random.default_rng(3)
    for i in rng.integers(0, scan.n, size=12):
        for X in rng.uniform(-128, 128, size=(5, 3)):
            p = A[i] @ np.append(X, 1.0)
            u, v, w = geometric_projection(scan, scan.betas[i], X)
            assert p[2] == pytest.approx(w, rel=1e-13)
            assert p[0] / p[2] == pytest.approx(u, abs=1e-9)
            assert p[1] / p[2] == pytest.approx(v, abs=1e-9)


def test_source_is_null_space_of_matrix():
    scan = synth.SCANS["tiny"]
    A = oracle.carm_matrices(scan)
    S = oracle.source_positions(A)
    for i, b in enumerate(scan.betas):
        expect = np.array([scan.sid * math.cos(b), scan.sid * math.sin(b), 0.0])
        np.testing.assert_allclose(S[i], expect, atol=1e-9)
        np.testing.assert_allclose(A[i] @ np.append(S[i], 1.0), 0.0, atol=1e-12)


def test_listing_column_major_indexing():
    """Listing 1 reads A column-major (A[0], A[1], A[2] multiply wx); the row-
    major matrices used here evaluate to the same (uw, vw, w)."""
    A = oracle.carm_matrices(synth.SCANS["tiny"])[7]
    Acm = A.T.reshape(-1)            # Acm[c*3 + r] = A[r, c]
    wx, wy, wz = 13.0, -41.0, 27.5
    uw = Acm[0] * wx + Acm[3] * wy + Acm[6] * wz + Acm[9]
    vw = Acm[1] * wx + Acm[4] * wy + Acm[7] * wz + Acm[10]
    w = Acm[2] * wx + Acm[5] * wy + Acm[8] * wz + Acm[11]
    np.testing.assert_allclose(A @ [wx, wy, wz, 1.0], [uw, vw, w], rtol=1e-15)


def test_exact_rational_hand_case():
    """A 2x2x2 volume and one 3x2 image with a hand-made matrix: every voxel
    value is computed in exact rational arithmetic from the definition."""
    img = np.array([[1, 2, 4], [8, 16, 32]], dtype=np.float32)
    A = np.array([[[1.0, 0.5, 0.25, 0.125],
                   [0.25, 0.0, 0.75, -0.5],
                   [0.0, 0.0, 0.5, 1.0]]])
    got = oracle.backproject(2, 1.0, (0.0, 0.0, 0.0), img[None], A)
    F = Fraction
    for z in range(2):
        for y in range(2):
            for x in range(2):
                uw = F(x) + F(1, 2) * y + F(1, 4) * z + F(1, 8)
                vw = F(1, 4) * x + F(3, 4) * z - F(1, 2)
                w = F(1, 2) * z + 1
                u, v = uw / w, vw / w
                iu, iv = math.floor(u), math.floor(v)
                fu, fv = u - iu, v - iv

                def P(j, k):
                    return F(int(img[k, j])) if 0 <= j < 3 and 0 <= k < 2 else F(0)
                fx = (1 - fv) * ((1 - fu) * P(iu, iv) + fu * P(iu + 1, iv)) + \
                    fv * ((1 - fu) * P(iu, iv + 1) + fu * P(iu + 1, iv + 1))
                assert got[z, y, x] == pytest.approx(float(fx / (w * w)), rel=1e-15, abs=1e-15)


def test_brute_force_geometric_backprojection():
    """Whole small volume: oracle vs per-voxel ray-plane projection + listing."""
    scan, vol = SMALL, synth.Volume(8)
    A = oracle.carm_matrices(scan)
    rng = np.random.default_rng(11)
    imgs = rng.standard_normal((scan.n, scan.isy, scan.isx)).astype(np.float32)
    got = oracle.backproject(vol.L, vol.R, vol.O, imgs, A)
    for z in range(vol.L):
        for y in range(vol.L):
            for x in range(vol.L):
                X = np.array(vol.O) + vol.R * np.array([x, y, z])
                acc = 0.0
                for i, b in enumerate(scan.betas):
                    u, v, w = geometric_projection(scan, b, X)
                    acc += listing_sample(imgs[i], u, v) / (w * w)
                assert got[z, y, x] == pytest.approx(acc, rel=1e-11, abs=1e-12)


def test_voxel_subset_matches_full_volume():
    scan, vol = SMALL, synth.Volume(8)
    A = oracle.carm_matrices(scan)
    imgs = np.random.default_rng(5).random((scan.n, scan.isy, scan.isx), dtype=np.float32)
    full = oracle.backproject(vol.L, vol.R, vol.O, imgs, A)
    idx = np.array([0, 7, 63, 64, 200, 511])
    np.testing.assert_array_equal(oracle.backproject_voxels(vol.L, vol.R, vol.O, imgs, A, idx),
                                  full.reshape(-1)[idx])


def test_constant_projections_closed_form():
    """p == c: every voxel seen inside [0,ISX-1]x[0,ISY-1] by all projections
    gets exactly c * sum_i (SID / depth_i)^2."""
    scan, vol = synth.SCANS["tiny"], synth.Volume(16)
    A = oracle.carm_matrices(scan)
    c = 0.75
    imgs = np.full((scan.n, scan.isy, scan.isx), c, dtype=np.float32)
    got = oracle.backproject(vol.L, vol.R, vol.O, imgs, A)
    checked = 0
    for z in range(0, vol.L, 3):
        for y in range(0, vol.L, 3):
            for x in range(vol.L):
                X = np.array(vol.O) + vol.R * np.array([x, y, z])
                tot, inside = 0.0, True
                for b in scan.betas:
                    u, v, w = geometric_projection(scan, b, X)
                    inside &= 0 <= u <= scan.isx - 1 and 0 <= v <= scan.isy - 1
                    tot += 1.0 / (w * w)
                if inside:
                    checked += 1
                    assert got[z, y, x] == pytest.approx(c * tot, rel=1e-12)
    assert checked > 500


def test_single_pixel_support_and_weights():
    """A unit pixel at (j, k): each voxel gets (1-|u-j|)+ (1-|v-k|)+ / w^2."""
    scan, vol = synth.Scan(n=1, isx=160, isy=120, pitch=7.68, beta0_deg=30.0), synth.Volume(16)
    j, k = 83, 57
    img = np.zeros((1, scan.isy, scan.isx), dtype=np.float32)
    img[0, k, j] = 1.0
    A = oracle.carm_matrices(scan)
    got = oracle.backproject(vol.L, vol.R, vol.O, img, A)
    nz = 0
    for z in range(vol.L):
        for y in range(vol.L):
            for x in range(vol.L):
                X = np.array(vol.O) + vol.R * np.array([x, y, z])
                u, v, w = geometric_projection(scan, scan.betas[0], X)
                e = max(0.0, 1 - abs(u - j)) * max(0.0, 1 - abs(v - k)) / (w * w)
                nz += e > 0
                assert got[z, y, x] == pytest.approx(e, abs=1e-12)
    assert nz > 0


def test_z_mirror_symmetry():
    """Images mirrored about the principal row reconstruct the z-mirrored volume."""
    scan, vol = synth.SCANS["tiny"], synth.Volume(16)
    A = oracle.carm_matrices(scan)
    imgs = np.random.default_rng(2).standard_normal((scan.n, scan.isy, scan.isx)).astype(np.float32)
    V = oracle.backproject(vol.L, vol.R, vol.O, imgs, A)
    Vm = oracle.backproject(vol.L, vol.R, vol.O, imgs[:, ::-1, :].copy(), A)
    np.testing.assert_allclose(Vm, V[::-1], rtol=1e-9, atol=1e-12 * np.abs(V).max())


def test_quarter_turn_relabels_the_volume():
    """Rotating the whole C-arm by 90 degrees about z (every source and
    detector) turns the reconstruction by 90 degrees: the voxel at world
    (x, y, z) of the rotated scan equals the voxel at (y, -x, z) of the
    original, i.e. V90[z, a, b] = V[z, L-1-b, a] on the centred grid."""
    base = synth.SCANS["tiny"]
    vol = synth.Volume(16)
    rot = synth.Scan(n=base.n, isx=base.isx, isy=base.isy, pitch=base.pitch, beta0_deg=base.beta0_deg + 90.0)
    imgs = np.random.default_rng(7).standard_normal((base.n, base.isy, base.isx)).astype(np.float32)
    V = oracle.backproject(vol.L, vol.R, vol.O, imgs, oracle.carm_matrices(base))
    V90 = oracle.backproject(vol.L, vol.R, vol.O, imgs, oracle.carm_matrices(rot))
    expect = V.transpose(0, 2, 1)[:, :, ::-1]
    np.testing.assert_allclose(V90, expect, rtol=1e-9, atol=1e-12 * np.abs(V).max())
    assert not np.allclose(V90, V, rtol=1e-3)          # the relabelling is not the identity here


def test_point_object_reconstructs_at_its_voxel():
    """A small sphere away from the isocenter, forward-projected by the
    analytic line integrals and reconstructed by FDK, peaks at the voxel
    nearest its centre."""
    scan, vol = synth.SCANS["train"], synth.Volume(32)
    A = oracle.carm_matrices(scan)
    idx = (20, 12, 18)                                  # (x, y, z) voxel indices
    X0 = [vol.O[k] + vol.R * idx[k] for k in range(3)]
    lines = oracle.ellipsoid_project(A, scan.isx, scan.isy, synth.sphere(tuple(X0), 5.0, 1.0))
    V = oracle.backproject(vol.L, vol.R, vol.O, oracle.fdk_filter(scan, lines).astype(np.float32), A)
    z, y, x = np.unravel_index(int(np.argmax(V)), V.shape)
    assert (x, y, z) == idx
    # sampled at its centre the reconstruction gives the sphere's density
    # (FDK's normalisation); the next voxel (8 mm away, outside) is near 0
    assert V[z, y, x] == pytest.approx(1.0, rel=0.1)
    assert np.sort(V.ravel())[-2] < 0.1


def test_linearity():
    scan, vol = synth.SCANS["tiny"], synth.Volume(12)
    A = oracle.carm_matrices(scan)
    rng = np.random.default_rng(4)
    p = (rng.integers(-512, 512, (scan.n, scan.isy, scan.isx)) / 256).astype(np.float32)
    q = (rng.integers(-512, 512, (scan.n, scan.isy, scan.isx)) / 256).astype(np.float32)
    comb = (2.0 * p - 3.0 * q).astype(np.float32)      # exact in float32
    Bp = oracle.backproject(vol.L, vol.R, vol.O, p, A)
    Bq = oracle.backproject(vol.L, vol.R, vol.O, q, A)
    Bc = oracle.backproject(vol.L, vol.R, vol.O, comb, A)
    np.testing.assert_allclose(Bc, 2 * Bp - 3 * Bq, atol=1e-11 * np.abs(Bc).max())


def test_adjoint_dot_product():
    """<B p, f> = <p, B^T f> for random p and f."""
    scan, vol = synth.SCANS["tiny"], synth.Volume(16)
    A = oracle.carm_matrices(scan)
    rng = np.random.default_rng(6)
    p = rng.standard_normal((scan.n, scan.isy, scan.isx)).astype(np.float32)
    f = rng.standard_normal((vol.L,) * 3)
    Bp = oracle.backproject(vol.L, vol.R, vol.O, p, A)
    Btf = oracle.adjoint(vol.L, vol.R, vol.O, f, A, scan.isx, scan.isy)
    lhs = float(np.sum(Bp * f))
    rhs = float(np.sum(p.astype(np.float64) * Btf))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_adjoint_of_unit_voxel():
    """B^T of a unit voxel is the bilinear footprint of its projection / w^2."""
    scan, vol = synth.Scan(n=2, isx=160, isy=120, pitch=7.68, beta0_deg=17.0), synth.Volume(8)
    A = oracle.carm_matrices(scan)
    f = np.zeros((8, 8, 8))
    f[5, 2, 6] = 1.0
    out = oracle.adjoint(vol.L, vol.R, vol.O, f, A, scan.isx, scan.isy)
    X = np.array(vol.O) + vol.R * np.array([6, 2, 5])
    for i, b in enumerate(scan.betas):
        u, v, w = geometric_projection(scan, b, X)
        expect = np.zeros((scan.isy, scan.isx))
        iu, iv = math.floor(u), math.floor(v)
        for (jj, kk) in [(iu, iv), (iu + 1, iv), (iu, iv + 1), (iu + 1, iv + 1)]:
            expect[kk, jj] = max(0, 1 - abs(u - jj)) * max(0, 1 - abs(v - kk)) / (w * w)
        np.testing.assert_allclose(out[i], expect, atol=1e-14)


# --------------------------------------------------------------------------
# Phantom line integrals and voxelisation.
def test_sphere_chord_lengths():
    scan = synth.SCANS["tiny"]
    A = oracle.carm_matrices(scan)[:3]
    cen, r, rho = np.array([10.0, -5.0, 3.0]), 40.0, 0.5
    out = oracle.ellipsoid_project(A, scan.isx, scan.isy, synth.sphere(cen, r, rho))
    for i in range(3):
        b = scan.betas[i]
        c, s = math.cos(b), math.sin(b)
        S = np.array([scan.sid * c, scan.sid * s, 0.0])
        Dc = S + scan.sdd * np.array([-c, -s, 0.0])
        for j in range(0, scan.isx, 7):
            for k in range(0, scan.isy, 5):
                P = Dc + (j - scan.cu) * scan.pitch * np.array([-s, c, 0.0]) + \
                    (k - scan.cv) * scan.pitch * np.array([0.0, 0.0, 1.0])
                dirn = (P - S) / np.linalg.norm(P - S)
                dist = np.linalg.norm(np.cross(cen - S, dirn))
                expect = rho * 2 * math.sqrt(r * r - dist * dist) if dist < r else 0.0
                assert out[i, k, j] == pytest.approx(expect, abs=1e-9)


def test_rotated_ellipsoid_by_ray_marching():
    """Line integral through a rotated ellipsoid vs dense sampling along the ray
    (a transposed rotation would change the answer)."""
    scan = synth.Scan(n=1, isx=160, isy=120, pitch=7.68, beta0_deg=40.0)
    A = oracle.carm_matrices(scan)
    ell = synth.ellipsoids(1, seed=9, scan=scan)
    ell[0, 0:3] = (5.0, -8.0, 6.0)
    ell[0, 3:6] = (60.0, 25.0, 12.0)
    out = oracle.ellipsoid_project(A, scan.isx, scan.isy, ell)
    Q = ell[0, 6:15].reshape(3, 3)
    assert not np.allclose(Q, Q.T)
    b = scan.betas[0]
    c, s = math.cos(b), math.sin(b)
    S = np.array([scan.sid * c, scan.sid * s, 0.0])
    Dc = S + scan.sdd * np.array([-c, -s, 0.0])
    t = np.linspace(scan.sid - 150, scan.sid + 150, 100001)
    dt = t[1] - t[0]
    hits = 0
    for j in range(72, 86):
        for k in range(55, 68):
            P = Dc + (j - scan.cu) * scan.pitch * np.array([-s, c, 0.0]) + \
                (k - scan.cv) * scan.pitch * np.array([0.0, 0.0, 1.0])
            dirn = (P - S) / np.linalg.norm(P - S)
            pts = S[None] + t[:, None] * dirn[None]
            loc = (pts - ell[0, 0:3]) @ Q / ell[0, 3:6]
            inside = np.sum(loc * loc, axis=1) <= 1.0
            expect = ell[0, 15] * inside.sum() * dt
            hits += expect > 0
            assert out[0, k, j] == pytest.approx(expect, abs=3 * dt * ell[0, 15])
    assert hits > 20


def test_voxelize_sphere_volume_and_axes():
    vol = synth.Volume(64)
    r = 50.0
    V = oracle.ellipsoid_voxelize(vol.L, vol.R, vol.O, synth.sphere((3.0, -2.0, 1.0), r, 1.0))
    assert V.sum() * vol.R ** 3 == pytest.approx(4 / 3 * math.pi * r ** 3, rel=0.01)
    # rotated ellipsoid: points just inside/outside along its first axis
    ell = synth.ellipsoids(1, seed=4, scan=synth.SCANS["tiny"])
    ell[0, 3:6] = (70.0, 20.0, 10.0)
    Q = ell[0, 6:15].reshape(3, 3)
    L, R = 3, 1.0
    for f, inside in [(0.97, True), (1.03, False)]:
        X = ell[0, 0:3] + f * 70.0 * Q[:, 0]
        O = X - R * np.array([1, 1, 1])       # voxel (1, 1, 1) sits at X
        got = oracle.ellipsoid_voxelize(L, R, O, ell)[1, 1, 1]
        assert (got > 0) == inside


# --------------------------------------------------------------------------
# FDK preprocessing.
def test_ramlak_frequency_response():
    """tau * sum_m h(m) e^{-i w m} = |w| / (2 pi tau): the band-limited ramp."""
    tau = 0.37
    M = 20001
    m = np.arange(-M, M + 1)
    h = np.array([oracle.ramlak(int(k), tau) for k in m])
    for w in (0.0, math.pi / 2, math.pi, 1.0):
        H = tau * np.sum(h * np.cos(w * m))
        assert H == pytest.approx(abs(w) / (2 * math.pi * tau), abs=2e-4 / tau)


def test_ramp_filter_is_linear_convolution():
    tau = 0.5
    rng = np.random.default_rng(8)
    x = rng.standard_normal((3, 2, 37))
    h = np.array([oracle.ramlak(int(k), tau) for k in range(-36, 37)])
    got = oracle.ramp_filter(x, tau)
    for r in range(3):
        for k in range(2):
            expect = tau * np.convolve(x[r, k], h, mode="full")[36:36 + 37]
            np.testing.assert_allclose(got[r, k], expect, rtol=1e-12, atol=1e-12)


def test_parker_conjugate_rays_sum_to_one():
    scan = synth.SCANS["full"]
    delta = 0.5 * (math.radians(scan.scan_deg) - math.pi)
    gmax = math.atan(scan.isx * scan.pitch / 2 / scan.sdd)
    assert delta > gmax
    rng = np.random.default_rng(1)
    n = 0
    for _ in range(2000):
        g = rng.uniform(-gmax, gmax)
        b = rng.uniform(0, math.pi + 2 * delta)
        bc = b + math.pi - 2 * g
        if bc > math.pi + 2 * delta:
            bc = b - math.pi - 2 * g
        if not (0 <= bc <= math.pi + 2 * delta):
            assert oracle.parker(b, g, delta) == pytest.approx(1.0, abs=1e-12)
            continue
        n += 1
        assert oracle.parker(b, g, delta) + oracle.parker(bc, -g, delta) == pytest.approx(1.0, abs=1e-12)
    assert n > 100


def test_conjugate_ray_convention_from_matrices():
    """Ray (b, g) and ray (b + pi - 2g, -g) are one line: each source projects
    onto the other's detector at fan angle -/+ g."""
    scan = synth.SCANS["full"]
    g = 0.1
    b1 = 0.3
    b2 = b1 + math.pi - 2 * g
    two = synth.Scan(n=2, isx=scan.isx, isy=scan.isy, pitch=scan.pitch,
                     scan_deg=math.degrees(b2 - b1), beta0_deg=math.degrees(b1))
    A = oracle.carm_matrices(two)
    S = oracle.source_positions(A)
    # S2 seen from projection 1, behind the detector plane: the ray through it
    p = A[0] @ np.append(S[1], 1.0)
    ut = (p[0] / p[2] - two.cu) * two.pitch
    assert math.atan(ut / two.sdd) == pytest.approx(g, abs=1e-12)
    p = A[1] @ np.append(S[0], 1.0)
    ut = (p[0] / p[2] - two.cu) * two.pitch
    assert math.atan(ut / two.sdd) == pytest.approx(-g, abs=1e-12)


def test_preweight_is_cosine_of_ray_angle_times_parker():
    """Cosine weight = cos of the angle between the central ray and the ray to
    the pixel (3-D geometry); with Parker on, the extra factor is the Parker
    weight at (beta_i - beta_0, fan angle of the column)."""
    scan = synth.Scan(n=5, isx=31, isy=23, pitch=12.3)
    ones = np.ones((scan.n, scan.isy, scan.isx))
    cosw = oracle.fdk_preweight(scan, ones, parker=False, scale=2.0)
    both = oracle.fdk_preweight(scan, ones, parker=True, scale=1.0)
    delta = 0.5 * (math.radians(scan.scan_deg) - math.pi)
    for i, b in enumerate(scan.betas):
        c, s = math.cos(b), math.sin(b)
        S = np.array([scan.sid * c, scan.sid * s, 0.0])
        d = np.array([-c, -s, 0.0])
        Dc = S + scan.sdd * d
        for k in range(0, scan.isy, 4):
            for j in range(0, scan.isx, 3):
                P = Dc + (j - scan.cu) * scan.pitch * np.array([-s, c, 0.0]) + \
                    (k - scan.cv) * scan.pitch * np.array([0.0, 0.0, 1.0])
                cos_ang = float((P - S) @ d) / np.linalg.norm(P - S)
                assert cosw[i, k, j] == pytest.approx(2.0 * cos_ang, rel=1e-13)
                fan = math.atan((j - scan.cu) * scan.pitch / scan.sdd)
                assert both[i, k, j] == pytest.approx(
                    cos_ang * oracle.parker(b - scan.betas[0], fan, delta), rel=1e-13, abs=1e-15)


def test_fdk_reconstructs_uniform_sphere_density():
    """Full chain (line integrals, cosine + Parker weights, ramp, backprojection)
    gives the sphere's density in its interior (FDK sanity, not parity)."""
    scan, vol = synth.SCANS["train"], synth.Volume(32)
    A = oracle.carm_matrices(scan)
    rho, r = 0.02, 60.0
    lines = oracle.ellipsoid_project(A, scan.isx, scan.isy, synth.sphere((0.0, 0.0, 0.0), r, rho))
    q = oracle.fdk_filter(scan, lines, parker=True)
    V = oracle.backproject(vol.L, vol.R, vol.O, q.astype(np.float32), A)
    zz, yy, xx = np.meshgrid(*(np.array(vol.O[0]) + vol.R * np.arange(vol.L),) * 3, indexing="ij")
    inner = (xx ** 2 + yy ** 2 + zz ** 2) < (0.6 * r) ** 2
    outer = (xx ** 2 + yy ** 2 + zz ** 2) > (1.4 * r) ** 2
    assert V[inner].mean() == pytest.approx(rho, rel=0.03)
    assert abs(V[outer & (np.abs(zz) < 40)].mean()) < 0.05 * rho


def test_row_filter_matches_correlation_and_adjoint():
    rng = np.random.default_rng(12)
    T, isx = 8, 29
    x = rng.standard_normal((4, isx))
    h = rng.standard_normal(T)
    y = oracle.row_filter_fwd(x, h)
    for r in range(4):
        pad = np.concatenate([np.zeros(T // 2), x[r], np.zeros(T)])
        expect = np.correlate(pad, h, mode="valid")[:isx]
        np.testing.assert_allclose(y[r], expect, rtol=1e-12, atol=1e-12)
    g = rng.standard_normal(y.shape)
    gin, gh = oracle.row_filter_bwd(x, h, g)
    assert float(np.sum(y * g)) == pytest.approx(float(np.sum(x * gin)), rel=1e-12)
    eps = 1e-6
    for t in range(T):
        hp = h.copy()
        hp[t] += eps
        fd = (np.sum(oracle.row_filter_fwd(x, hp) * g) - np.sum(y * g)) / eps
        assert gh[t] == pytest.approx(fd, rel=1e-5, abs=1e-7)


# --------------------------------------------------------------------------
# Numbers the paper prints that the measurement code depends on.
def test_paper_metric_facts():
    facts = json.load(open(os.path.join(GOLDEN, "paper_facts.json")))
    f = facts["realtime_goal"]
    updates = f["L"] ** 3 * f["n_proj"]
    assert updates / f["seconds"] / 1e9 == pytest.approx(f["gups"], abs=0.005)
    f = facts["volume_traffic"]
    per_sweep = f["L"] ** 3 * f["bytes_per_voxel_update"]
    assert per_sweep / 2 ** 30 == pytest.approx(f["per_sweep_gb"], rel=1e-12)
    assert per_sweep * f["n_proj"] / 2 ** 30 == pytest.approx(f["all_proj_gb"], rel=1e-12)
    f = facts["projection_stack"]
    assert f["n_proj"] * f["isx"] * f["isy"] * 4 / 1e9 == pytest.approx(f["gb"], abs=0.05)


def test_error_measures_closed_forms():
    """Sect. 7.2's PSNR and the relative L2 error on cases with closed forms:
    a reference spanning [2, 10] (M = 8) and a reconstruction off by a
    constant 0.01 give 10 log10(64 / 1e-4) = 58.06 dB; a reconstruction off
    by alternating +-0.5 on a reference of constant 4 gives rel-L2 1/8."""
    R = np.linspace(2.0, 10.0, 1001)
    assert oracle.psnr(R + 0.01, R) == pytest.approx(10.0 * math.log10(64.0 / 1e-4), abs=1e-9)
    assert oracle.psnr(R, R) == float("inf")
    # the PSNR does not depend on where the reference's range sits
    assert oracle.psnr(R + 100.01, R + 100.0) == pytest.approx(oracle.psnr(R + 0.01, R), abs=1e-6)
    ref = np.full(1000, 4.0)
    got = ref + 0.5 * np.where(np.arange(1000) % 2 == 0, 1.0, -1.0)
    assert oracle.rel_l2(got, ref) == pytest.approx(0.125, rel=1e-12)
