"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: a closed form,
a brute-force evaluation, an invariant, an independent algebraic form, or the
numbers the paper prints.  Sizes are tiny so the whole file runs in seconds.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import prism_oracle as O
from paper_1702_01904_gb300 import specimens

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_grid(n=64, cell=6.4, f=1, H=3, dz=2.0, ds=2, alpha=20.0, aa=0.5):
    return dict(nx=n, ny=n, cell_x=cell, cell_y=cell, n_slices=H, dz=dz, kv=300.0, f=f,
                downsample=ds, aa_frac=aa, alpha_mrad=alpha)


def rand_potential(grid, seed, amp=150.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return (amp * rng.random((grid["n_slices"], grid["ny"], grid["nx"]))).astype(np.float32)


DET = dict(start_mrad=0.0, step_mrad=1.0, nbins=120)
PROBE = dict(alpha_mrad=20.0, c1=0.0, c3=0.0)


# ------------------------------------------------------------------ constants
def test_wavelength_textbook_form():
    # lambda[A] = 12.2643 / sqrt(V (1 + 0.978476e-6 V)), the common closed form with rounded constants
    for kv in (80.0, 200.0, 300.0):
        v = kv * 1e3
        ref = 12.2643 / math.sqrt(v * (1.0 + 0.978476e-6 * v))
        assert abs(O.wavelength(kv) - ref) / ref < 2e-5
    # the 300 kV value quoted for the workloads: 0.01969 A
    assert abs(O.wavelength(300.0) - 0.01969) < 5e-6


def test_sigma_alternative_form():
    # sigma = (2 pi / (lambda V)) (m0 c^2 + eV) / (2 m0 c^2 + eV): algebraically equal to 2 pi m e lambda / h^2
    for kv in (80.0, 300.0):
        v = kv * 1e3
        mc2 = O.M_ELECTRON * O.C_LIGHT ** 2 / O.Q_ELECTRON  # in eV
        ref = 2 * math.pi / (O.wavelength(kv) * v) * (mc2 + v) / (2 * mc2 + v)
        assert abs(O.interaction_constant(kv) - ref) / ref < 1e-12
    assert abs(O.interaction_constant(300.0) - 6.526e-4) < 1e-6


# ------------------------------------------------------------------ P1: FFT convention
def test_fft_matches_bruteforce_dft():
    rng = np.random.Generator(np.random.PCG64(11))
    a = rng.normal(size=(16, 16)) + 1j * rng.normal(size=(16, 16))
    k = np.arange(16)
    w = np.exp(-2j * np.pi * np.outer(k, k) / 16)
    brute = np.zeros_like(a)
    for ky in range(16):
        for kx in range(16):
            brute[ky, kx] = np.sum(a * w[ky][:, None] * w[kx][None, :])
    assert np.max(np.abs(O.fft2(a) - brute)) < 1e-12 * np.max(np.abs(brute))
    assert np.max(np.abs(O.ifft2(brute) - a)) < 1e-12
    # signed indices: k >= n/2 maps to k - n
    assert list(O.signed_freq_index(8)) == [0, 1, 2, 3, -4, -3, -2, -1]


# ------------------------------------------------------------------ P2: norm conservation
def test_norm_conserved_without_aa_and_nonincreasing_with_aa():
    g = small_grid(H=6)
    v = rand_potential(g, 2)
    psi = O.plane_wave(64, 64, 6.4, 6.4, 0.0, 0.0)
    t = O.transmission(v, 300.0)
    assert np.max(np.abs(np.abs(t) - 1.0)) < 1e-14
    p_free = O.propagator(64, 64, 6.4, 6.4, 300.0, 2.0, aa_frac=None)
    p_aa = O.propagator(64, 64, 6.4, 6.4, 300.0, 2.0, aa_frac=0.5)
    n0 = np.sum(np.abs(psi) ** 2)
    a, b = psi, psi
    last = n0
    for p in range(6):
        a = O.multislice(a, t[p:p + 1], p_free)
        b = O.multislice(b, t[p:p + 1], p_aa)
        assert abs(np.sum(np.abs(a) ** 2) - n0) < 1e-12 * n0
        nb = np.sum(np.abs(b) ** 2)
        assert nb <= last * (1 + 1e-13)
        last = nb
    assert last < n0 * 0.9999  # random potential scatters beyond the aperture


# ------------------------------------------------------------------ Fresnel closed forms
def gaussian(n, cell, c, w2):
    x = np.arange(n) * (cell / n) - c
    r2 = x[None, :] ** 2 + x[:, None] ** 2
    return np.exp(-r2 / (2 * w2))


def test_free_space_gaussian_beam_closed_form():
    # d psi/dz = (i lambda / 4 pi) lap psi: a Gaussian of width w becomes
    # (w^2 / W^2) exp(-r^2 / 2W^2) with W^2 = w^2 + i lambda z / (2 pi).
    n, cell, w = 128, 20.0, 0.8
    lam = O.wavelength(300.0)
    H, dz = 8, 25.0
    psi0 = gaussian(n, cell, 10.0, w * w)
    t = np.ones((H, n, n), dtype=complex)
    prop = O.propagator(n, n, cell, cell, 300.0, dz, aa_frac=None)
    out = O.multislice(psi0, t, prop)
    W2 = w * w + 1j * lam * H * dz / (2 * math.pi)
    ref = (w * w / W2) * gaussian(n, cell, 10.0, W2)
    assert np.max(np.abs(out - ref)) < 1e-10


def test_transmit_then_propagate_order_tilt_walkoff():
    # One slice with t = exp(2 pi i g.r): transmit-then-propagate moves the beam by lambda z g
    # and multiplies by exp(-i pi lambda z g^2) exp(2 pi i g.r).  The other order would not move it.
    n, cell, w = 128, 20.0, 0.8
    lam = O.wavelength(300.0)
    z = 200.0
    g = 10.0 / cell
    x = np.arange(n) * (cell / n)
    tilt = np.exp(2j * math.pi * g * x)[None, :] * np.ones((n, 1))
    psi0 = gaussian(n, cell, 10.0, w * w)
    prop = O.propagator(n, n, cell, cell, 300.0, z, aa_frac=None)
    out = O.multislice(psi0, tilt[None], prop)
    W2 = w * w + 1j * lam * z / (2 * math.pi)
    shift = lam * z * g
    xs = x - 10.0 - shift
    ys = x - 10.0
    free = (w * w / W2) * np.exp(-(xs[None, :] ** 2 + ys[:, None] ** 2) / (2 * W2))
    ref = np.exp(-1j * math.pi * lam * z * g * g) * tilt * free
    assert np.max(np.abs(out - ref)) < 1e-10


@pytest.mark.parametrize("axis", [1, 0])
def test_weak_phase_grating_contrast_sign(axis):
    # Weak phase object V = eps cos(2 pi g x) under a plane wave, one slice, then free flight z.
    # To first order in sigma eps, t = 1 + i sigma eps cos(2 pi g x); the two diffracted beams at
    # +-g each pick up exp(-i pi lambda z g^2), so the exit intensity is
    #   I(x) = 1 + 2 sigma eps sin(pi lambda z g^2) cos(2 pi g x) + O((sigma eps)^2).
    # The sign of the contrast term is the sign of the transmission phase (the propagator's sign is
    # fixed by the Gaussian-beam pin): exp(-i sigma V) would flip it.  The exit wave comes from the
    # oracle's own S-matrix path (the q = 0 beam at full resolution), so the whole composition of
    # transmission, propagator and slice step is what is checked.
    n, cell, kg, z = 64, 16.0, 4, 200.0
    lam = O.wavelength(300.0)
    sig = O.interaction_constant(300.0)
    g = kg / cell
    x = np.arange(n) * (cell / n)
    phase_q = math.pi * lam * z * g * g
    assert math.sin(phase_q) > 0.5  # a clearly positive contrast transfer at this z
    grid = dict(nx=n, ny=n, cell_x=cell, cell_y=cell, n_slices=1, dz=z, kv=300.0, f=1,
                downsample=1, aa_frac=0.5, alpha_mrad=20.0)
    residuals = []
    for eps in (30.0, 15.0):  # sigma * eps = 0.0196 and 0.0098
        line = eps * np.cos(2 * math.pi * g * x)
        v = np.broadcast_to(line[None, :] if axis == 1 else line[:, None], (n, n))[None].copy()
        S, _, _ = O.smatrix_build(v, grid, beams=(np.array([0]), np.array([0])))
        inten = np.abs(S[0]) ** 2
        model = 1.0 + 2.0 * sig * eps * math.sin(phase_q) * np.cos(2 * math.pi * g * x)
        model = np.broadcast_to(model[None, :] if axis == 1 else model[:, None], (n, n))
        res = float(np.max(np.abs(inten - model)))
        assert res <= 2.0 * (sig * eps) ** 2, (eps, res)
        # the bright fringe sits on the potential's maximum (x = 0) for a positive potential
        assert inten[0, 0] > 1.0 + sig * eps * math.sin(phase_q)
        residuals.append(res)
    # the residual is second order: halving eps quarters it
    assert 3.0 < residuals[0] / residuals[1] < 5.0


# ------------------------------------------------------------------ beam set
def gauss_circle_count(r2):
    r = int(math.isqrt(int(math.floor(r2)))) + 1
    return sum(1 for m in range(-r, r + 1) for n in range(-r, r + 1) if m * m + n * n <= r2)


@pytest.mark.parametrize("cell,n,f", [(16.0, 256, 4), (50.0, 1024, 8), (32.0, 512, 8), (6.4, 64, 1)])
def test_beam_set_is_gauss_circle(cell, n, f):
    lam = O.wavelength(300.0)
    r = 0.020 / (f * lam / cell)          # aperture radius in units of the beam lattice step
    m, nn = O.beam_set(n, n, cell, cell, 300.0, f, 20.0)
    assert len(m) == gauss_circle_count(r * r)
    assert len(set(zip(m.tolist(), nn.tolist()))) == len(m)


def test_beam_counts_of_the_two_main_workloads():
    # lattice-point counts of the 20 mrad aperture on the f*dq lattice at 300 kV
    assert len(O.beam_set(256, 256, 16.0, 16.0, 300.0, 4, 20.0)[0]) == gauss_circle_count((0.02 / (4 * O.wavelength(300.0) / 16.0)) ** 2)
    assert len(O.beam_set(256, 256, 16.0, 16.0, 300.0, 4, 20.0)[0]) == 49
    assert len(O.beam_set(1024, 1024, 50.0, 50.0, 300.0, 8, 20.0)[0]) == 129


# ------------------------------------------------------------------ P3: empty sample multislice
def test_empty_sample_multislice_is_aperture_count():
    g = small_grid(n=64, cell=8.0, H=4)
    v = np.zeros((4, 64, 64), np.float32)
    out = O.multislice_probe(v, g, PROBE, DET, 1.3, 2.9)
    lam = O.wavelength(300.0)
    counts = np.zeros(DET["nbins"])
    total = 0
    for ky in range(-32, 32):
        for kx in range(-32, 32):
            k2 = kx * kx + ky * ky
            if (lam / 8.0) ** 2 * k2 <= 0.02 ** 2 * (1 + 1e-12):
                total += 1
                counts[int(1000 * lam * math.sqrt(k2) / 8.0)] += 1
    assert np.max(np.abs(out - counts / total)) < 1e-12
    assert abs(out.sum() - 1.0) < 1e-12


def test_uniform_potential_is_global_phase():
    # P8: V = const only adds a phase; intensities equal the empty sample
    g = small_grid(n=64, cell=8.0, H=3, f=2)
    v0 = np.zeros((3, 64, 64), np.float32)
    v1 = np.full((3, 64, 64), 123.0, np.float32)
    a = O.multislice_probe(v0, g, PROBE, DET, 2.0, 3.0)
    b = O.multislice_probe(v1, g, PROBE, DET, 2.0, 3.0)
    assert np.max(np.abs(a - b)) < 1e-12
    S0, m, n = O.smatrix_build(v0, g)
    S1, _, _ = O.smatrix_build(v1, g)
    xs, ys = np.array([0.4, 5.1]), np.array([7.7, 1.2])
    assert np.max(np.abs(O.prism_scan(S0, m, n, g, PROBE, DET, xs, ys)
                         - O.prism_scan(S1, m, n, g, PROBE, DET, xs, ys))) < 1e-12


# ------------------------------------------------------------------ S-matrix closed form
def test_smatrix_empty_sample_closed_form():
    # with V = 0 each stored beam is its plane wave times exp(-i pi lambda |q|^2 H dz), at amplitude 1
    g = small_grid(n=64, cell=8.0, H=3, f=2)
    S, m, n = O.smatrix_build(np.zeros((3, 64, 64), np.float32), g)
    lam = O.wavelength(300.0)
    x = np.arange(32) * (8.0 / 32)
    for b in range(len(m)):
        qx, qy = m[b] * 2 / 8.0, n[b] * 2 / 8.0
        ref = np.exp(2j * math.pi * (qx * x[None, :] + qy * x[:, None])) \
            * np.exp(-1j * math.pi * lam * 3 * 2.0 * (qx * qx + qy * qy))
        assert np.max(np.abs(S[b] - ref)) < 1e-12


# ------------------------------------------------------------------ P4: f = 1 equals multislice
@pytest.mark.parametrize("ds", [1, 2])
def test_prism_f1_equals_multislice(ds):
    g = small_grid(n=64, cell=6.4, H=3, f=1, ds=ds)
    v = rand_potential(g, 4)
    S, m, n = O.smatrix_build(v, g)
    xs, ys = np.array([0.0, 1.37, 5.9]), np.array([0.0, 4.21, 6.3])
    pr = O.prism_scan(S, m, n, g, PROBE, DET, xs, ys)
    ms = O.multislice_scan(v, g, PROBE, DET, xs, ys)
    assert np.max(np.abs(pr - ms)) < 1e-12
    assert np.all(np.abs(pr.sum(1) - 1.0) < 0.05)


# ------------------------------------------------------------------ P5: crop off at f > 1
def test_prism_crop_off_equals_multislice_of_periodic_probe():
    g = small_grid(n=64, cell=8.0, H=3, f=2)
    v = rand_potential(g, 5)
    S, m, n = O.smatrix_build(v, g)
    x0, y0 = 2.3, 5.55
    pr = O.prism_scan(S, m, n, g, PROBE, DET, np.array([x0]), np.array([y0]), full_window=True)[0]
    a = O.probe_coefficients(m, n, g, PROBE, x0, y0)
    psi = sum(a[b] * O.plane_wave(64, 64, 8.0, 8.0, m[b] * 2 / 8.0, n[b] * 2 / 8.0) for b in range(len(m)))
    psi = O.multislice(psi, O.transmission(v, 300.0), O.propagator(64, 64, 8.0, 8.0, 300.0, 2.0))
    spec = np.fft.fft2(psi)                      # full-res spectrum; AA keeps it inside the N/2 square
    inten = np.abs(spec) ** 2 / (64 ** 4 * np.sum(np.abs(a) ** 2))
    lam = O.wavelength(300.0)
    ref = np.zeros(DET["nbins"])
    k = O.signed_freq_index(64)
    for iy in range(64):
        for ix in range(64):
            th = 1000 * lam * math.hypot(k[ix] / 8.0, k[iy] / 8.0)
            if th < DET["nbins"]:
                ref[int(th)] += inten[iy, ix]
    assert np.max(np.abs(pr - ref)) < 1e-12


def test_prism_direct_linearity_equals_smatrix_scan():
    g = small_grid(n=64, cell=8.0, H=3, f=4)
    v = rand_potential(g, 6)
    S, m, n = O.smatrix_build(v, g)
    for x0, y0 in [(0.0, 0.0), (3.3, 7.9), (7.99, 0.26)]:
        a = O.prism_scan(S, m, n, g, PROBE, DET, np.array([x0]), np.array([y0]))[0]
        b = O.prism_probe_direct(v, g, PROBE, DET, x0, y0)
        assert np.max(np.abs(a - b)) < 1e-12


# ------------------------------------------------------------------ P6: one slice, brute force window
def test_single_slice_window_bruteforce():
    n, cell, f = 64, 8.0, 4
    g = small_grid(n=n, cell=cell, H=1, f=f, dz=0.0)
    v = rand_potential(g, 7)
    S, m, nb = O.smatrix_build(v, g)
    lam = O.wavelength(300.0)
    sig = O.interaction_constant(300.0)
    x0, y0 = 6.71, 0.4
    pr = O.prism_scan(S, m, nb, g, PROBE, DET, np.array([x0]), np.array([y0]))[0]
    # direct: periodic probe, transmit, AA-filter (dz = 0), half-resolution grid, window by loops
    xr = np.arange(n) * (cell / n)
    psi = np.zeros((n, n), complex)
    norm = 0.0
    for b in range(len(m)):
        qx, qy = m[b] * f / cell, nb[b] * f / cell
        c = np.exp(-2j * math.pi * (qx * x0 + qy * y0))
        norm += abs(c) ** 2
        psi += c * np.exp(2j * math.pi * (qx * xr[None, :] + qy * xr[:, None]))
    psi = psi * np.exp(1j * sig * v[0].astype(float))
    k = O.signed_freq_index(n)
    spec = np.fft.fft2(psi)
    half = np.zeros((n // 2, n // 2), complex)
    for iy in range(n):
        for ix in range(n):
            if -n // 4 <= k[iy] < n // 4 and -n // 4 <= k[ix] < n // 4:
                if (k[ix] / cell) ** 2 + (k[iy] / cell) ** 2 < (0.25 * n / cell) ** 2:
                    half[k[iy] % (n // 2), k[ix] % (n // 2)] = spec[iy, ix]
    low = np.fft.ifft2(half) / 4.0
    nd = n // 2
    nw = nd // f
    px = cell / nd
    sx = int(math.floor(x0 / px + 0.5)) - nw // 2
    sy = int(math.floor(y0 / px + 0.5)) - nw // 2
    win = np.zeros((nw, nw), complex)
    for v_ in range(nw):
        for u in range(nw):
            win[v_, u] = low[(sy + v_) % nd, (sx + u) % nd]
    ref = np.zeros(DET["nbins"])
    kw = O.signed_freq_index(nw)
    for ky in range(nw):
        for kx in range(nw):
            s = 0j
            for v_ in range(nw):
                for u in range(nw):
                    s += win[v_, u] * np.exp(-2j * math.pi * (kx * u + ky * v_) / nw)
            th = 1000 * lam * math.hypot(kw[kx] * f / cell, kw[ky] * f / cell)
            if th < DET["nbins"]:
                ref[int(th)] += abs(s) ** 2 / (nw ** 4 * norm)
    assert np.max(np.abs(pr - ref)) < 1e-12


# ------------------------------------------------------------------ P7: shift equivariance
def test_shift_equivariance():
    g = small_grid(n=64, cell=8.0, H=2, f=2)
    v = rand_potential(g, 8)
    kx, ky = 3, 5
    v2 = np.roll(v, (2 * ky, 2 * kx), axis=(1, 2))
    S, m, n = O.smatrix_build(v, g)
    S2, _, _ = O.smatrix_build(v2, g)
    px = 8.0 / 32
    xs, ys = np.array([1.0, 2.6]), np.array([0.5, 6.1])
    a = O.prism_scan(S, m, n, g, PROBE, DET, xs, ys)
    b = O.prism_scan(S2, m, n, g, PROBE, DET, xs + kx * px, ys + ky * px)
    assert np.max(np.abs(a - b)) < 1e-12


# ------------------------------------------------------------------ P10: beam orthogonality on the window
def test_empty_sample_window_has_one_pixel_per_beam():
    g = small_grid(n=64, cell=8.0, H=2, f=2)
    S, m, n = O.smatrix_build(np.zeros((2, 64, 64), np.float32), g)
    out = O.prism_scan(S, m, n, g, PROBE, DET, np.array([1.7]), np.array([3.2]))[0]
    lam = O.wavelength(300.0)
    ref = np.zeros(DET["nbins"])
    for b in range(len(m)):
        ref[int(1000 * lam * 2 * math.sqrt(m[b] ** 2 + n[b] ** 2) / 8.0)] += 1.0 / len(m)
    assert np.max(np.abs(out - ref)) < 1e-12


# ------------------------------------------------------------------ window origin and detector
def test_window_origin_centres_nearest_pixel_and_wraps():
    px = 0.5
    assert O.window_origin(3 * px + 0.2, 16.0, 32, 8) == (3 - 4) % 32
    assert O.window_origin(3 * px + 0.3, 16.0, 32, 8) == (4 - 4) % 32
    assert O.window_origin(0.0, 16.0, 32, 8) == 28
    assert O.window_origin(3.74 * px, 16.0, 32, 8) == 0
    assert O.window_origin(-0.3 * px, 16.0, 32, 8) == 28
    assert O.window_origin(31.6 * px, 16.0, 32, 8) == 28


def test_detector_bins_basic():
    lam = O.wavelength(300.0)
    det = dict(start_mrad=5.0, step_mrad=2.0, nbins=3)
    q = np.array([0.0, 6.0, 7.5, 10.5, 11.5]) / (1000 * lam)
    b = O.detector_bins(q, np.zeros_like(q), lam, det)
    assert list(b) == [-1, 0, 1, 2, -1]


# ------------------------------------------------------------------ P9: the paper's cost model
def test_cost_model_printed_speedups():
    gold = json.load(open(os.path.join(GOLDEN, "cost_model_speedups.json")))
    for f, printed in zip(gold["f"], gold["printed_speedup"]):
        r = O.speedup_ratio(gold["H"], gold["P"], gold["B"], f)
        assert abs(r - printed) / printed <= gold["printed_rounding_rel"]
        # the ratio is the large-N limit of Eq. TimeMulti / Eq. TimePRISM
        N = 2 ** 24
        full = O.cost_multislice(gold["H"], gold["P"], N) / O.cost_prism(gold["H"], gold["P"], N, gold["B"], f)
        assert abs(full - r) / r < 1e-4
    assert [round(O.speedup_ratio(40, 1e5, 1e4, f), 1) for f in (2, 4, 8, 16)] == [0.5, 7.8, 108.8, 1152.8]


# ------------------------------------------------------------------ inputs
def test_specimen_potential_peak():
    spec = specimens.simple_cubic(8.0, 2.0, 29)
    v = specimens.project_potential(spec, 64, 64, 4, 2.0)
    # atoms on pixel centres, 2 A apart: peak = V0 Z^0.7 plus small neighbour tails
    peak = specimens.V0_VA * 29 ** 0.7
    assert abs(v.max() - peak) / peak < 1e-3
    assert v.shape == (4, 64, 64) and v.dtype == np.float32


# ------------------------------------------------------------------ aberrations
def test_chi_matches_wave_aberration_in_angles():
    # chi = (2 pi / lambda) W(theta), W = C1 theta^2 / 2 + C3 theta^4 / 4, theta = lambda |q|
    lam = O.wavelength(300.0)
    for q in (0.1, 0.7, 1.3):
        th = lam * q
        ref = 2 * math.pi / lam * (35.0 * th ** 2 / 2 + 1.2e5 * th ** 4 / 4)
        assert abs(O.chi(q * q, lam, 35.0, 1.2e5) - ref) < 1e-12 * abs(ref)


def test_defocus_minus_thickness_refocuses_at_exit():
    # exp(-i chi) with C1 = -z and the Fresnel factor exp(-i pi lambda q^2 z) cancel: the exit wave of an
    # empty sample is the in-focus probe.
    g = small_grid(n=64, cell=8.0, H=4, dz=12.5)
    z = 4 * 12.5
    x0, y0 = 3.1, 4.7
    psi0 = O.ifft2(O.probe_spectrum(g, dict(alpha_mrad=20.0, c1=-z, c3=0.0), x0, y0))
    t = np.ones((4, 64, 64), complex)
    out = O.multislice(psi0, t, O.propagator(64, 64, 8.0, 8.0, 300.0, 12.5))
    focused = O.ifft2(O.probe_spectrum(g, dict(alpha_mrad=20.0, c1=0.0, c3=0.0), x0, y0))
    assert np.max(np.abs(out - focused)) < 1e-12
    # a probe defocused the other way is not focused
    psi1 = O.ifft2(O.probe_spectrum(g, dict(alpha_mrad=20.0, c1=z, c3=0.0), x0, y0))
    out1 = O.multislice(psi1, t, O.propagator(64, 64, 8.0, 8.0, 300.0, 12.5))
    assert np.max(np.abs(out1 - focused)) > 1e-3


# ------------------------------------------------------------------ probe tilt, CBED, frozen phonons
def test_tilted_empty_sample_counts_shifted_aperture():
    # a tilted probe is the aperture disc centred on q_t = theta / lambda; with V = 0 each of its
    # pixels keeps its intensity and lands in the bin of its own |q| (lattice-point count)
    g = small_grid(n=64, cell=8.0, H=3)
    lam = O.wavelength(300.0)
    probe = dict(alpha_mrad=12.0, c1=0.0, c3=0.0, tilt_x=0.015, tilt_y=-0.008)
    out = O.multislice_probe(np.zeros((3, 64, 64), np.float32), g, probe, DET, 2.5, 1.0)
    counts = np.zeros(DET["nbins"])
    total = 0
    for ky in range(-32, 32):
        for kx in range(-32, 32):
            dx, dy = kx / 8.0 - 0.015 / lam, ky / 8.0 + 0.008 / lam
            if (lam * dx) ** 2 + (lam * dy) ** 2 <= 0.012 ** 2 * (1 + 1e-12):
                total += 1
                counts[int(1000 * lam * math.sqrt(kx * kx + ky * ky) / 8.0)] += 1
    assert total > 10
    assert np.max(np.abs(out - counts / total)) < 1e-12


def test_tilt_shift_recentres_exit_probe():
    # coefficients at r0 - h tan(theta): the tilted probe walks h*theta through the cell and exits
    # centred on r0 (to O(theta^3)); dropping the shift would leave it h tan(theta) away
    # (256^2 over 24 A: anti-aliasing cutoff 52 mrad, above the 45 mrad reached by the tilted aperture)
    g = small_grid(n=256, cell=24.0, H=5, dz=20.0)
    h = 100.0
    th = 0.02
    probe = dict(alpha_mrad=25.0, c1=0.0, c3=0.0, tilt_x=th, tilt_y=0.0)
    x0, y0 = 12.0, 12.0
    psi = O.ifft2(O.probe_spectrum(g, probe, x0, y0))
    x = np.arange(256) * (24.0 / 256)
    inten = np.abs(psi) ** 2
    assert abs(float(np.sum(inten * x[None, :]) / inten.sum()) - (x0 - h * math.tan(th))) < 0.1
    psi = O.multislice(psi, np.ones((5, 256, 256), complex), O.propagator(256, 256, 24.0, 24.0, 300.0, 20.0))
    inten = np.abs(psi) ** 2
    cx = float(np.sum(inten * x[None, :]) / inten.sum())
    cy = float(np.sum(inten * x[:, None]) / inten.sum())
    assert abs(cx - x0) < 0.1 and abs(cy - y0) < 0.1  # Airy tails in a periodic box bias the centroid slightly
    assert abs(h * math.tan(th) - 2.0) < 0.01  # the shift being tested is 2 A


def test_prism_f1_equals_multislice_with_tilt_and_aberrations():
    g = small_grid(n=64, cell=6.4, H=3, f=1, ds=2, alpha=28.0)
    v = rand_potential(g, 12)
    probe = dict(alpha_mrad=18.0, c1=40.0, c3=1.0e4, tilt_x=0.006, tilt_y=0.004)
    S, m, n = O.smatrix_build(v, g)
    xs, ys = np.array([0.3, 4.1]), np.array([5.5, 2.0])
    pr = O.prism_scan(S, m, n, g, probe, DET, xs, ys)
    ms = O.multislice_scan(v, g, probe, DET, xs, ys)
    assert np.max(np.abs(pr - ms)) < 1e-12


def test_cbed_empty_sample_one_pixel_per_beam_and_bins_consistent():
    g = small_grid(n=64, cell=8.0, H=2, f=2)
    S, m, n = O.smatrix_build(np.zeros((2, 64, 64), np.float32), g)
    cb = O.prism_cbed(S, m, n, g, PROBE, np.array([1.1]), np.array([6.3]))[0]
    ref = np.zeros((16, 16))
    for b in range(len(m)):
        ref[n[b] % 16, m[b] % 16] = 1.0 / len(m)
    assert np.max(np.abs(cb - ref)) < 1e-12
    v = rand_potential(g, 13)
    S, m, n = O.smatrix_build(v, g)
    xs, ys = np.array([0.7, 3.9]), np.array([2.2, 7.1])
    cb = O.prism_cbed(S, m, n, g, PROBE, xs, ys)
    bins = O.window_bins(g, DET, 16, 16, (2, 8.0), (2, 8.0))
    for p in range(2):
        assert np.allclose(O.bin_sum(cb[p], bins, DET["nbins"]), O.prism_scan(S, m, n, g, PROBE, DET, xs[p:p + 1], ys[p:p + 1])[0], atol=1e-14)


def test_frozen_phonon_average():
    g = small_grid(n=64, cell=8.0, H=2, f=2)
    v1, v2 = rand_potential(g, 14), rand_potential(g, 15)
    xs, ys = np.array([1.0]), np.array([2.0])
    same = O.frozen_phonon_scan([v1, v1, v1], g, PROBE, DET, xs, ys)
    S, m, n = O.smatrix_build(v1, g)
    single = O.prism_scan(S, m, n, g, PROBE, DET, xs, ys)
    assert np.max(np.abs(same - single)) < 1e-15
    S2, _, _ = O.smatrix_build(v2, g)
    mix = O.frozen_phonon_scan([v1, v2], g, PROBE, DET, xs, ys)
    assert np.max(np.abs(mix - 0.5 * (single + O.prism_scan(S2, m, n, g, PROBE, DET, xs, ys)))) < 1e-15


# ------------------------------------------------------------------ separate interpolation factors f_x, f_y
def test_rectangular_beam_lattice_is_the_even_rows_of_the_square_one():
    # f_y = 2 f: the beams (m, n) with (m f / c)^2 + (2 n f / c)^2 inside the aperture are exactly
    # the square-lattice beams (m, n') with n' even, n = n' / 2
    for n_px, cell, f in [(256, 16.0, 4), (512, 32.0, 4), (128, 12.8, 1)]:
        m, n = O.beam_set(n_px, n_px, cell, cell, 300.0, f, 20.0, 2 * f)
        ms, ns = O.beam_set(n_px, n_px, cell, cell, 300.0, f, 20.0)
        want = {(int(a), int(b) // 2) for a, b in zip(ms, ns) if b % 2 == 0}
        assert set(zip(m.tolist(), n.tolist())) == want and len(m) == len(want)
    # f_x = 2 f_y: the even columns of the f_y lattice
    for n_px, cell, fy in [(256, 16.0, 2), (512, 50.0, 4)]:
        m, n = O.beam_set(n_px, n_px, cell, cell, 300.0, 2 * fy, 20.0, fy)
        ms, ns = O.beam_set(n_px, n_px, cell, cell, 300.0, fy, 20.0)
        want = {(int(a) // 2, int(b)) for a, b in zip(ms, ns) if a % 2 == 0}
        assert set(zip(m.tolist(), n.tolist())) == want and len(m) == len(want)


def test_single_slice_rectangular_window_bruteforce():
    # one slice, dz = 0, f_x = 2, f_y = 4: periodic probe on the (2 dq, 4 dq) lattice, transmit,
    # anti-aliasing filter, half-resolution grid, a 16 x 8 window by loops, its DFT by loops
    n, cell, fx, fy = 64, 8.0, 2, 4
    g = dict(small_grid(n=n, cell=cell, H=1, f=fx, dz=0.0), f_y=fy)
    v = rand_potential(g, 17)
    S, m, nb = O.smatrix_build(v, g)
    lam = O.wavelength(300.0)
    sig = O.interaction_constant(300.0)
    x0, y0 = 3.61, 7.7
    pr = O.prism_scan(S, m, nb, g, PROBE, DET, np.array([x0]), np.array([y0]))[0]
    xr = np.arange(n) * (cell / n)
    psi = np.zeros((n, n), complex)
    norm = 0.0
    for b in range(len(m)):
        qx, qy = m[b] * fx / cell, nb[b] * fy / cell
        c = np.exp(-2j * math.pi * (qx * x0 + qy * y0))
        norm += abs(c) ** 2
        psi += c * np.exp(2j * math.pi * (qx * xr[None, :] + qy * xr[:, None]))
    psi = psi * np.exp(1j * sig * v[0].astype(float))
    k = O.signed_freq_index(n)
    spec = np.fft.fft2(psi)
    half = np.zeros((n // 2, n // 2), complex)
    for iy in range(n):
        for ix in range(n):
            if -n // 4 <= k[iy] < n // 4 and -n // 4 <= k[ix] < n // 4:
                if (k[ix] / cell) ** 2 + (k[iy] / cell) ** 2 < (0.25 * n / cell) ** 2:
                    half[k[iy] % (n // 2), k[ix] % (n // 2)] = spec[iy, ix]
    low = np.fft.ifft2(half) / 4.0
    nd = n // 2
    nwx, nwy = nd // fx, nd // fy
    px = cell / nd
    sx = int(math.floor(x0 / px + 0.5)) - nwx // 2
    sy = int(math.floor(y0 / px + 0.5)) - nwy // 2
    win = np.zeros((nwy, nwx), complex)
    for v_ in range(nwy):
        for u in range(nwx):
            win[v_, u] = low[(sy + v_) % nd, (sx + u) % nd]
    ref = np.zeros(DET["nbins"])
    kwx, kwy = O.signed_freq_index(nwx), O.signed_freq_index(nwy)
    for ky in range(nwy):
        for kx in range(nwx):
            s = 0j
            for v_ in range(nwy):
                for u in range(nwx):
                    s += win[v_, u] * np.exp(-2j * math.pi * (kx * u / nwx + ky * v_ / nwy))
            th = 1000 * lam * math.hypot(kwx[kx] * fx / cell, kwy[ky] * fy / cell)
            if th < DET["nbins"]:
                ref[int(th)] += abs(s) ** 2 / ((nwx * nwy) ** 2 * norm)
    assert np.max(np.abs(pr - ref)) < 1e-12


def test_rectangular_crop_off_equals_multislice_of_periodic_probe():
    g = dict(small_grid(n=64, cell=8.0, H=3, f=1), f_y=2)
    v = rand_potential(g, 18)
    S, m, n = O.smatrix_build(v, g)
    x0, y0 = 5.1, 1.35
    pr = O.prism_scan(S, m, n, g, PROBE, DET, np.array([x0]), np.array([y0]), full_window=True)[0]
    a = O.probe_coefficients(m, n, g, PROBE, x0, y0)
    psi = sum(a[b] * O.plane_wave(64, 64, 8.0, 8.0, m[b] / 8.0, n[b] * 2 / 8.0) for b in range(len(m)))
    psi = O.multislice(psi, O.transmission(v, 300.0), O.propagator(64, 64, 8.0, 8.0, 300.0, 2.0))
    inten = np.abs(np.fft.fft2(psi)) ** 2 / (64 ** 4 * np.sum(np.abs(a) ** 2))
    lam = O.wavelength(300.0)
    ref = np.zeros(DET["nbins"])
    k = O.signed_freq_index(64)
    for iy in range(64):
        for ix in range(64):
            th = 1000 * lam * math.hypot(k[ix] / 8.0, k[iy] / 8.0)
            if th < DET["nbins"]:
                ref[int(th)] += inten[iy, ix]
    assert np.max(np.abs(pr - ref)) < 1e-12


def test_rectangular_window_empty_sample_one_pixel_per_beam_and_linearity():
    g = dict(small_grid(n=64, cell=8.0, H=2, f=4), f_y=2)
    S, m, n = O.smatrix_build(np.zeros((2, 64, 64), np.float32), g)
    out = O.prism_scan(S, m, n, g, PROBE, DET, np.array([2.2]), np.array([6.9]))[0]
    lam = O.wavelength(300.0)
    ref = np.zeros(DET["nbins"])
    for b in range(len(m)):
        ref[int(1000 * lam * math.hypot(m[b] * 4 / 8.0, n[b] * 2 / 8.0))] += 1.0 / len(m)
    assert np.max(np.abs(out - ref)) < 1e-12
    v = rand_potential(g, 19)
    S, m, n = O.smatrix_build(v, g)
    for x0, y0 in [(0.0, 0.0), (6.3, 2.9)]:
        a = O.prism_scan(S, m, n, g, PROBE, DET, np.array([x0]), np.array([y0]))[0]
        assert np.max(np.abs(a - O.prism_probe_direct(v, g, PROBE, DET, x0, y0))) < 1e-12


def test_periodic_probe_wave_is_the_plane_wave_sum():
    # the spectrum form of sum_b a_b exp(2 pi i q_b.r) against the plane waves evaluated one by one,
    # on a rectangular grid with f_x != f_y (a transposed or mis-scaled bin would fail)
    rng = np.random.Generator(np.random.PCG64(12))
    nx, ny, cx, cy, f, fy = 48, 32, 6.0, 4.0, 3, 2
    m, n = O.beam_set(nx, ny, cx, cy, 300.0, f, 40.0, fy)
    assert len(m) > 6 and len(set(zip(m, n))) == len(m)
    a = rng.normal(size=len(m)) + 1j * rng.normal(size=len(m))
    x = np.arange(nx) * (cx / nx)
    y = np.arange(ny) * (cy / ny)
    brute = np.zeros((ny, nx), dtype=complex)
    for b in range(len(m)):
        brute += a[b] * np.exp(2j * math.pi * (m[b] * f / cx * x[None, :] + n[b] * fy / cy * y[:, None]))
    assert np.max(np.abs(O.periodic_probe_wave(a, m, n, nx, ny, f, fy) - brute)) < 1e-12 * len(m)


# ------------------------------------------------------------------ identities the CUDA path relies on
def test_first_slice_shift_theorem():
    # the first row transform of a plane wave times t_0 is the row transform of t_0 shifted by the
    # plane wave's column index, times its y phase (the build makes the first slice this way)
    rng = np.random.Generator(np.random.PCG64(3))
    nx, ny, m, n, f, fy = 32, 16, -3, 2, 2, 1
    t0 = np.exp(1j * rng.random((ny, nx)) * 2.0)
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    psi = np.exp(2j * np.pi * (m * f * x / nx + n * fy * y / ny))
    direct = np.fft.fft(psi * t0, axis=1)
    T0 = np.fft.fft(t0, axis=1)
    kx = np.arange(nx)
    shifted = T0[:, (kx - m * f) % nx] * np.exp(2j * np.pi * (n * fy * np.arange(ny) / ny))[:, None]
    assert np.max(np.abs(direct - shifted)) < 1e-12 * nx


def test_half_resolution_storage_is_every_second_sample():
    # a wave band-limited to |k| < N/4 (what the anti-aliasing aperture leaves) has its inner-square
    # Fourier crop, inverse-transformed at N/2 and divided by 4, equal to its even real-space samples
    rng = np.random.Generator(np.random.PCG64(4))
    n = 32
    k = np.fft.fftfreq(n, 1.0 / n)
    band = (np.abs(k)[:, None] < n // 4) & (np.abs(k)[None, :] < n // 4)
    spec = (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) * band
    wave = np.fft.ifft2(spec)
    crop = O.fourier_crop_half(wave)
    assert np.max(np.abs(crop - wave[::2, ::2])) < 1e-13
