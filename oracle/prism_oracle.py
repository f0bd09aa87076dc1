"""FP64 CPU oracle for PRISM STEM simulation and plain multislice (Ophus 2017).

TEST INFRASTRUCTURE.  Only the tests, the package's smoke check and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA path: nothing here imports the package, and the package never
imports this.  It is deliberately plain and slow: NumPy float64/complex128,
``numpy.fft`` as the FFT primitive, loops where the paper loops.

Each function names the passage of the paper it follows ("Multislice" section,
"PRISM Algorithm" section, equations by their labels in the paper).

Readings of points the paper leaves open (all are listed in the design notes):
  O1  lambda, sigma from CODATA constants (relativistic); the paper gives no numbers.
  O2  FFT: forward unnormalised exp(-2 pi i k x / N), inverse with 1/N^2 (numpy).
      Frequencies q = k / cell for the signed integer k in FFT order.
  O3  Each slice: transmit, then propagate -- also after the last slice (Eq. Multislice).
  O4  Anti-aliasing aperture |q| < aa_frac * q_nyquist (strict), q_nyquist =
      min(nx/(2 cx), ny/(2 cy)), applied inside the propagator of every slice.
  O5  Beam set: lambda*|q_mn| <= alpha (inclusive, with a 1e-12 relative slack), beams
      ordered n (y index) ascending, then m ascending.
  O6  Window origin s = floor(x0 / px' + 1/2) - Nw/2 (mod N'), px' = cell / N'.
  O7  Intensities in units of the total incident probe intensity.
  O8  Detector bin b = floor((1000 lambda |q| - start) / step), kept if 0 <= b < nbins.

Parity status: every function below is pinned by the oracle self-tests
(closed forms, brute force, invariants and the paper's printed cost-model
values); PRISM-vs-multislice *accuracy* at f > 1 is an approximation of the
method and is reported, not gated.
"""
from __future__ import annotations

import math

import numpy as np

# CODATA 2018 (SI)
H_PLANCK = 6.62607015e-34      # J s (exact)
M_ELECTRON = 9.1093837015e-31  # kg
Q_ELECTRON = 1.602176634e-19   # C (exact)
C_LIGHT = 299792458.0          # m/s (exact)
BEAM_SLACK = 1e-12             # relative slack of the inclusive aperture tests


# ------------------------------------------------------------------ physics
def wavelength(kv: float) -> float:
    """Relativistic electron wavelength in Angstrom (symbol lambda in Eq. Schrodinger)."""
    ev = Q_ELECTRON * (kv * 1e3)
    p2 = 2.0 * M_ELECTRON * ev * (1.0 + ev / (2.0 * M_ELECTRON * C_LIGHT * C_LIGHT))
    return H_PLANCK / math.sqrt(p2) * 1e10


def interaction_constant(kv: float) -> float:
    """sigma = 2 pi m e lambda / h^2 in rad/(V*Angstrom), m the relativistic mass (Eq. Schrodinger)."""
    ev = Q_ELECTRON * (kv * 1e3)
    m = M_ELECTRON + ev / (C_LIGHT * C_LIGHT)
    lam_m = wavelength(kv) * 1e-10
    return 2.0 * math.pi * m * Q_ELECTRON * lam_m / (H_PLANCK * H_PLANCK) * 1e-10


# ------------------------------------------------------------------ grids
def signed_freq_index(n: int) -> np.ndarray:
    """Integer frequency indices in FFT order: 0..n/2-1, -n/2..-1."""
    return np.concatenate([np.arange(0, (n + 1) // 2), np.arange(-(n // 2), 0)]).astype(np.int64)


def freq_grid(nx, ny, cell_x, cell_y):
    """(qx[ny,nx], qy[ny,nx]) in 1/Angstrom, q = k / cell (reading O2)."""
    qx = signed_freq_index(nx).astype(np.float64) / cell_x
    qy = signed_freq_index(ny).astype(np.float64) / cell_y
    return np.broadcast_to(qx[None, :], (ny, nx)), np.broadcast_to(qy[:, None], (ny, nx))


def fft2(a):
    """Forward 2-D DFT, exp(-2 pi i k.x/N), unnormalised (reading O2)."""
    return np.fft.fft2(a)


def ifft2(a):
    """Inverse 2-D DFT with the 1/(nx ny) factor (reading O2)."""
    return np.fft.ifft2(a)


# ------------------------------------------------------- multislice pieces
def transmission(v_slices, kv):
    """t_p(r) = exp(i sigma V_p(r))  (Multislice section, transmission operator)."""
    return np.exp(1j * interaction_constant(kv) * np.asarray(v_slices, dtype=np.float64))


def aa_mask(nx, ny, cell_x, cell_y, aa_frac):
    """Anti-aliasing aperture |q| < aa_frac * q_nyquist (PRISM Algorithm section; reading O4).

    ``aa_frac=None`` disables the aperture (used only by the norm-conservation pin).
    """
    if aa_frac is None:
        return np.ones((ny, nx), dtype=bool)
    qx, qy = freq_grid(nx, ny, cell_x, cell_y)
    q_nyq = min(0.5 * nx / cell_x, 0.5 * ny / cell_y)
    q_aa = aa_frac * q_nyq
    return qx * qx + qy * qy < q_aa * q_aa


def propagator(nx, ny, cell_x, cell_y, kv, dz, aa_frac=0.5):
    """P(q) = exp(-i pi lambda |q|^2 t), times the AA aperture (Multislice section, Fresnel operator)."""
    lam = wavelength(kv)
    qx, qy = freq_grid(nx, ny, cell_x, cell_y)
    q2 = qx * qx + qy * qy
    return np.exp(-1j * math.pi * lam * dz * q2) * aa_mask(nx, ny, cell_x, cell_y, aa_frac)


def multislice(psi, trans, props):
    """Eq. Multislice applied slice by slice: psi <- F^-1{ F{psi t_p} P_p }, p = 0..H-1.

    ``props`` is one propagator (uniform slices) or a list with one per slice.
    The propagation after the last slice is included (reading O3).
    """
    psi = np.asarray(psi, dtype=np.complex128)
    for p in range(trans.shape[0]):
        prop = props[p] if isinstance(props, (list, tuple)) else props
        psi = ifft2(fft2(psi * trans[p]) * prop)
    return psi


def slice_propagators(grid):
    dzs = grid.get("slice_dz")
    if dzs is None:
        return propagator(grid["nx"], grid["ny"], grid["cell_x"], grid["cell_y"], grid["kv"],
                          grid["dz"], grid.get("aa_frac", 0.5))
    return [propagator(grid["nx"], grid["ny"], grid["cell_x"], grid["cell_y"], grid["kv"],
                       float(d), grid.get("aa_frac", 0.5)) for d in dzs]


# ------------------------------------------------------------- PRISM pieces
def inside_aperture(qx, qy, lam, alpha_rad):
    """A(q) = 1 where lambda |q| <= alpha (aperture function, PRISM Algorithm section; reading O5)."""
    ax = lam * qx
    ay = lam * qy
    return ax * ax + ay * ay <= alpha_rad * alpha_rad * (1.0 + BEAM_SLACK)


def interpolation_factors(grid):
    """(f_x, f_y): the interpolation factor along x and along y (PRISM Algorithm section allows a
    different factor per axis; "f_y" absent or 0 means f_y = f)."""
    f = grid["f"]
    return f, (grid.get("f_y") or f)


def beam_set(nx, ny, cell_x, cell_y, kv, f, alpha_mrad, f_y=None):
    """Plane-wave indices (m, n): q_mn = (m f_x / cx, n f_y / cy) with lambda |q_mn| <= alpha_max
    (PRISM Algorithm section, plane-wave set; f_y = f unless given).  Returns int arrays m, n
    ordered n-major.
    """
    fy = f if not f_y else f_y
    lam = wavelength(kv)
    alpha = alpha_mrad * 1e-3
    mmax = int(math.floor(alpha / (lam * f / cell_x))) + 1
    nmax = int(math.floor(alpha / (lam * fy / cell_y))) + 1
    ms, ns = [], []
    for n in range(-nmax, nmax + 1):
        for m in range(-mmax, mmax + 1):
            qx = float(m * f) / cell_x
            qy = float(n * fy) / cell_y
            if inside_aperture(qx, qy, lam, alpha):
                ms.append(m)
                ns.append(n)
    return np.array(ms, dtype=np.int64), np.array(ns, dtype=np.int64)


def plane_wave(nx, ny, cell_x, cell_y, qx, qy):
    """psi(r) = exp(2 pi i q.r) at pixel centres r = (ix cx/nx, iy cy/ny)."""
    x = np.arange(nx, dtype=np.float64) * (cell_x / nx)
    y = np.arange(ny, dtype=np.float64) * (cell_y / ny)
    return np.exp(2j * math.pi * (qx * x[None, :] + qy * y[:, None]))


def fourier_crop_half(psi):
    """Keep the inner ny/2 x nx/2 frequencies, k in [-n/4, n/4), and return the real-space wave on
    the half-size grid with the plane-wave amplitude kept at 1 (the x4 storage saving the PRISM
    Algorithm section attributes to the anti-aliasing aperture)."""
    ny, nx = psi.shape
    big = fft2(psi)
    iy = np.r_[0:ny // 4, ny - ny // 4:ny]
    ix = np.r_[0:nx // 4, nx - nx // 4:nx]
    return ifft2(big[np.ix_(iy, ix)]) / 4.0


def smatrix_build(v_slices, grid, beams=None):
    """Compact S-matrix (PRISM Algorithm section, Fig. 1c): multislice of every plane wave in the
    f-subsampled aperture, stored in real space, optionally at half resolution per axis.

    Returns (S [B][ny'][nx'] complex128, m, n).
    """
    nx, ny, cx, cy = grid["nx"], grid["ny"], grid["cell_x"], grid["cell_y"]
    f, fy = interpolation_factors(grid)
    m, n = beam_set(nx, ny, cx, cy, grid["kv"], f, grid["alpha_mrad"], fy) if beams is None else beams
    trans = transmission(v_slices, grid["kv"])
    props = slice_propagators(grid)
    ds = grid.get("downsample", 2)
    out = []
    for b in range(len(m)):
        psi = plane_wave(nx, ny, cx, cy, float(m[b] * f) / cx, float(n[b] * fy) / cy)
        psi = multislice(psi, trans, props)
        out.append(fourier_crop_half(psi) if ds == 2 else psi)
    return np.array(out), m, n


def chi(q2, lam, c1, c3):
    """Aberration phase chi(q) = pi lambda q^2 C1 + (pi/2) lambda^3 q^4 C3 (PRISM Algorithm section)."""
    return math.pi * lam * q2 * c1 + 0.5 * math.pi * lam ** 3 * q2 * q2 * c3


def cell_height(grid):
    """Total thickness h of the simulation cell (sum of the slice thicknesses)."""
    dzs = grid.get("slice_dz")
    return float(grid["dz"]) * grid["n_slices"] if dzs is None else float(np.sum(dzs))


def tilt_terms(grid, probe):
    """Probe tilt (PRISM Algorithm section): the aperture and chi are centred on q_t = theta / lambda
    (the probe centre moved away from q = 0), and the coefficients use r0 - h tan(theta), which
    brings the tilted probe back to the centre of the cut-out region at the exit surface."""
    lam = wavelength(grid["kv"])
    tx, ty = probe.get("tilt_x", 0.0), probe.get("tilt_y", 0.0)
    h = cell_height(grid)
    return tx / lam, ty / lam, h * math.tan(tx), h * math.tan(ty)


def probe_coefficients(m, n, grid, probe, x0, y0):
    """alpha_mn(r0) = A(q - q_t) exp(-i chi(q - q_t)) exp(-2 pi i q.(r0 - h tan theta))
    (PRISM Algorithm section, coefficients and tilt)."""
    lam = wavelength(grid["kv"])
    f, fy = interpolation_factors(grid)
    qtx, qty, sx, sy = tilt_terms(grid, probe)
    qx = (m * f).astype(np.float64) / grid["cell_x"]
    qy = (n * fy).astype(np.float64) / grid["cell_y"]
    dqx = qx - qtx
    dqy = qy - qty
    a = inside_aperture(dqx, dqy, lam, probe["alpha_mrad"] * 1e-3)
    q2 = dqx * dqx + dqy * dqy
    return a * np.exp(-1j * chi(q2, lam, probe.get("c1", 0.0), probe.get("c3", 0.0))) \
        * np.exp(-2j * math.pi * (qx * (x0 - sx) + qy * (y0 - sy)))


def window_origin(x0, cell, n_ds, nw):
    """First pixel of the Nw-wide window around x0 on the stored grid (Eq. RegionBounds; reading O6)."""
    px = cell / n_ds
    return (int(math.floor(x0 / px + 0.5)) - nw // 2) % n_ds


def detector_bins(qx, qy, lam, det):
    """Annular bin index of each pixel, -1 outside (Fig. 1f virtual detectors; reading O8)."""
    theta = 1000.0 * lam * np.sqrt(qx * qx + qy * qy)
    b = np.floor((theta - det["start_mrad"]) / det["step_mrad"]).astype(np.int64)
    return np.where((b >= 0) & (b < det["nbins"]), b, -1)


def bin_sum(intensity, bins, nbins):
    out = np.zeros(nbins, dtype=np.float64)
    sel = bins >= 0
    np.add.at(out, bins[sel], intensity[sel])
    return out


def window_bins(grid, det, nwx, nwy, spacing_x, spacing_y):
    lam = wavelength(grid["kv"])
    qx = (signed_freq_index(nwx).astype(np.float64) * spacing_x[0]) / spacing_x[1]
    qy = (signed_freq_index(nwy).astype(np.float64) * spacing_y[0]) / spacing_y[1]
    return detector_bins(qx[None, :], qy[:, None], lam, det)


def prism_scan(S, m, n, grid, probe, det, x0s, y0s, full_window=False):
    """Probe scan (PRISM Algorithm section, Fig. 1d-f, Eq. PRISMfinal and Eq. RegionBounds).

    For each probe: coefficients, window of the stored grid around r0 (wrapped), beam sum,
    window FFT, |.|^2 in units of incident intensity, annular bins.
    ``full_window`` replaces the d/f window by the whole stored grid (crop off).
    Returns [P][nbins] float64.
    """
    nb, nyd, nxd = S.shape
    f, fy = interpolation_factors(grid)
    if full_window:
        nwx, nwy = nxd, nyd
        bins = window_bins(grid, det, nwx, nwy, (1, grid["cell_x"]), (1, grid["cell_y"]))
    else:
        nwx, nwy = nxd // f, nyd // fy
        bins = window_bins(grid, det, nwx, nwy, (f, grid["cell_x"]), (fy, grid["cell_y"]))
    out = np.zeros((len(x0s), det["nbins"]))
    for p in range(len(x0s)):
        a = probe_coefficients(m, n, grid, probe, x0s[p], y0s[p])
        sx = window_origin(x0s[p], grid["cell_x"], nxd, nwx)
        sy = window_origin(y0s[p], grid["cell_y"], nyd, nwy)
        iy = (sy + np.arange(nwy)) % nyd
        ix = (sx + np.arange(nwx)) % nxd
        win = S[:, iy[:, None], ix[None, :]]
        psi = np.tensordot(a, win, axes=(0, 0))
        norm = float(np.sum(np.abs(a) ** 2))
        inten = np.abs(fft2(psi)) ** 2 / ((nwx * nwy) ** 2 * norm)
        out[p] = bin_sum(inten, bins, det["nbins"])
    return out


def prism_cbed(S, m, n, grid, probe, x0s, y0s):
    """Full diffraction pattern of each probe's window (Fig. 1f, "full probe diffraction pattern"):
    |FFT_Nw(psi)|^2 in units of the incident intensity, window frequencies in FFT order.
    Returns [P][nw_y][nw_x] float64."""
    nb, nyd, nxd = S.shape
    f, fy = interpolation_factors(grid)
    nwx, nwy = nxd // f, nyd // fy
    out = np.zeros((len(x0s), nwy, nwx))
    for p in range(len(x0s)):
        a = probe_coefficients(m, n, grid, probe, x0s[p], y0s[p])
        sx = window_origin(x0s[p], grid["cell_x"], nxd, nwx)
        sy = window_origin(y0s[p], grid["cell_y"], nyd, nwy)
        win = S[:, ((sy + np.arange(nwy)) % nyd)[:, None], ((sx + np.arange(nwx)) % nxd)[None, :]]
        psi = np.tensordot(a, win, axes=(0, 0))
        norm = float(np.sum(np.abs(a) ** 2))
        out[p] = np.abs(fft2(psi)) ** 2 / ((nwx * nwy) ** 2 * norm) if norm > 0 else 0.0
    return out


def frozen_phonon_scan(v_configs, grid, probe, det, x0s, y0s):
    """Frozen-phonon average (Simulation and Analysis Implementation section): the PRISM result of
    each displaced-atom configuration, summed incoherently with equal weights."""
    acc = None
    for v in v_configs:
        S, m, n = smatrix_build(v, grid)
        r = prism_scan(S, m, n, grid, probe, det, x0s, y0s)
        acc = r if acc is None else acc + r
    return acc / len(v_configs)


def periodic_probe_wave(a, m, n, nx, ny, f, fy):
    """sum_b a_b exp(2 pi i q_b.r) on the grid, q_b = (m_b f / cx, n_b f_y / cy).

    At the pixel centres r = (ix cx/nx, iy cy/ny) each plane wave is exp(2 pi i (m_b f ix / nx +
    n_b f_y iy / ny)), the inverse-DFT basis function of the integer frequency (m_b f, n_b f_y).  So
    the sum is the inverse 2-D DFT of a spectrum holding nx ny a_b at that frequency's FFT bin
    (distinct beams occupy distinct bins).
    """
    spec = np.zeros((ny, nx), dtype=np.complex128)
    spec[(n * fy) % ny, (m * f) % nx] = np.asarray(a) * (nx * ny)
    return ifft2(spec)


def prism_probe_direct(v_slices, grid, probe, det, x0, y0):
    """One PRISM probe by linearity of Eq. PRISMfinal, without the S-matrix.

    sum_b alpha_b S_b = multislice( sum_b alpha_b exp(2 pi i q_b.r) ), so a probe's PRISM result
    is one multislice of its d/f-periodic incident wave, stored as the S-matrix would be, then the
    same window, FFT and bins.  Cost: one multislice per probe, usable at any grid size.
    """
    nx, ny, cx, cy = grid["nx"], grid["ny"], grid["cell_x"], grid["cell_y"]
    f, fy = interpolation_factors(grid)
    m, n = beam_set(nx, ny, cx, cy, grid["kv"], f, grid["alpha_mrad"], fy)
    a = probe_coefficients(m, n, grid, probe, x0, y0)
    psi = periodic_probe_wave(a, m, n, nx, ny, f, fy)
    psi = multislice(psi, transmission(v_slices, grid["kv"]), slice_propagators(grid))
    if grid.get("downsample", 2) == 2:
        psi = fourier_crop_half(psi)
    nyd, nxd = psi.shape
    nwx, nwy = nxd // f, nyd // fy
    sx = window_origin(x0, cx, nxd, nwx)
    sy = window_origin(y0, cy, nyd, nwy)
    win = psi[((sy + np.arange(nwy)) % nyd)[:, None], ((sx + np.arange(nwx)) % nxd)[None, :]]
    norm = float(np.sum(np.abs(a) ** 2))
    inten = np.abs(fft2(win)) ** 2 / ((nwx * nwy) ** 2 * norm)
    bins = window_bins(grid, det, nwx, nwy, (f, cx), (fy, cy))
    return bin_sum(inten, bins, det["nbins"])


# ------------------------------------------------------- multislice baseline
def probe_spectrum(grid, probe, x0, y0):
    """Psi0(q) = A(q - q_t) exp(-i chi(q - q_t)) exp(-2 pi i q.(r0 - h tan theta)) on the full
    Fourier grid (the same probe definition as the PRISM coefficients)."""
    lam = wavelength(grid["kv"])
    qtx, qty, sx, sy = tilt_terms(grid, probe)
    qx, qy = freq_grid(grid["nx"], grid["ny"], grid["cell_x"], grid["cell_y"])
    dqx = qx - qtx
    dqy = qy - qty
    a = inside_aperture(dqx, dqy, lam, probe["alpha_mrad"] * 1e-3)
    q2 = dqx * dqx + dqy * dqy
    return a * np.exp(-1j * chi(q2, lam, probe.get("c1", 0.0), probe.get("c3", 0.0))) \
        * np.exp(-2j * math.pi * (qx * (x0 - sx) + qy * (y0 - sy)))


def multislice_probe(v_slices, grid, probe, det, x0, y0, trans=None, props=None):
    """Conventional STEM multislice for one probe (Multislice section): probe -> H slices ->
    far-field |Psi|^2 / sum|Psi0|^2 -> annular bins."""
    psi0q = probe_spectrum(grid, probe, x0, y0)
    trans = transmission(v_slices, grid["kv"]) if trans is None else trans
    props = slice_propagators(grid) if props is None else props
    psi = multislice(ifft2(psi0q), trans, props)
    inten = np.abs(fft2(psi)) ** 2 / float(np.sum(np.abs(psi0q) ** 2))
    qx, qy = freq_grid(grid["nx"], grid["ny"], grid["cell_x"], grid["cell_y"])
    bins = detector_bins(qx, qy, wavelength(grid["kv"]), det)
    return bin_sum(inten, bins, det["nbins"])


def multislice_scan(v_slices, grid, probe, det, x0s, y0s):
    trans = transmission(v_slices, grid["kv"])
    props = slice_propagators(grid)
    return np.array([multislice_probe(v_slices, grid, probe, det, x0s[i], y0s[i], trans, props)
                     for i in range(len(x0s))])


# ------------------------------------------------------------ cost model
def cost_multislice(H, P, N):
    """Eq. TimeMulti: T_multi = H P (6 N log2 N + 2 N^2)."""
    return H * P * (6.0 * N * math.log2(N) + 2.0 * N * N)


def cost_prism(H, P, N, B, f):
    """Eq. TimePRISM: T_PRISM = (H B / f^2)(6 N log2 N + 2 N^2) + P B N^2 / (4 f^4)."""
    return H * B / f ** 2 * (6.0 * N * math.log2(N) + 2.0 * N * N) + P * B * N * N / (4.0 * f ** 4)


def speedup_ratio(H, P, B, f):
    """Eq. TimeRatio (large-N limit): 8 H P f^4 / (B (8 H f^2 + P))."""
    return 8.0 * H * P * f ** 4 / (B * (8.0 * H * f ** 2 + P))


# ------------------------------------------------------------- metrics
def rel_l2_per_image(test, ref):
    """Relative L2 error of each detector image ([P][nbins] -> [nbins])."""
    num = np.sqrt(np.sum((np.asarray(test, np.float64) - ref) ** 2, axis=0))
    den = np.sqrt(np.sum(np.asarray(ref) ** 2, axis=0))
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(den > 0, num / den, np.where(num == 0, 0.0, np.inf))


def one_minus_r2(a, b):
    """1 - R^2 between two images (Results section's error estimate)."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    if a.std() == 0 or b.std() == 0:
        return float("nan")
    return 1.0 - float(np.corrcoef(a, b)[0, 1]) ** 2
