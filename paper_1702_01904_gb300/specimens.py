"""Seeded synthetic specimens, workload shapes and scan geometries.

This module produces *inputs* only: atom coordinates, the projected potential
slices V_p(r) (V*Angstrom, float32) that a STEM simulation consumes, and the
probe positions of a raster scan.  It holds none of the simulation method's
arithmetic (no transmission, propagation, beam set, FFT or detector math), so
both the CUDA path and the FP64 oracle can take their inputs from here.

Stand-in for the paper's samples: the paper projects Kirkland atomic
potentials of a Pt decahedron on amorphous carbon (Results, Fig. 3/4); those
coordinates and the Kirkland tables are not available, so every atom here is a
2-D Gaussian of width ``SIGMA_G`` and peak ``V0_VA * Z**0.7``, summed over the
periodic images that lie within ``CUTOFF_SIGMAS`` widths of a pixel.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

V0_VA = 25.0          # V*Angstrom: peak projected potential of a Z=1 atom
SIGMA_G = 0.3         # Angstrom: Gaussian width of one atom's projected potential
CUTOFF_SIGMAS = 5.0   # contributions beyond 5 sigma of every periodic image are dropped


@dataclass
class Specimen:
    """Atoms in an orthorhombic cell; z runs along the beam from 0 (entrance)."""
    xyz: np.ndarray            # [n, 3] float64, Angstrom
    z_number: np.ndarray       # [n] int
    cell: tuple                # (cx, cy, cz) Angstrom
    note: str = ""


@dataclass
class Workload:
    """One simulation job: specimen, sampling and scan (all inputs)."""
    name: str
    nx: int
    ny: int
    cell_x: float
    cell_y: float
    n_slices: int
    dz: float
    kv: float
    f: int
    alpha_mrad: float
    scan_px: int
    scan_py: int
    scan_step: float
    det_start_mrad: float = 0.0
    det_step_mrad: float = 1.0
    det_nbins: int = 100
    downsample: int = 2
    aa_frac: float = 0.5
    c1: float = 0.0
    c3: float = 0.0
    specimen: Specimen | None = field(default=None, repr=False)

    def scan_positions(self):
        """Probe positions x0 = i*step, y0 = j*step, row-major [py][px] (Angstrom)."""
        xs = np.arange(self.scan_px, dtype=np.float64) * self.scan_step
        ys = np.arange(self.scan_py, dtype=np.float64) * self.scan_step
        y0, x0 = np.meshgrid(ys, xs, indexing="ij")
        return np.ascontiguousarray(x0.ravel()), np.ascontiguousarray(y0.ravel())

    def potential(self) -> np.ndarray:
        return project_potential(self.specimen, self.nx, self.ny, self.n_slices, self.dz)


# ---------------------------------------------------------------- specimens
def simple_cubic(cell=16.0, a=2.0, z_number=29) -> Specimen:
    """Simple-cubic crystal, atoms at (i a, j a, (k + 1/2) a): one plane per slice of thickness a."""
    n = int(round(cell / a))
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    xyz = np.stack([i.ravel() * a, j.ravel() * a, (k.ravel() + 0.5) * a], axis=1).astype(np.float64)
    return Specimen(xyz, np.full(len(xyz), z_number, dtype=np.int64), (cell, cell, cell),
                    note=f"simple cubic a={a} Z={z_number}")


def random_packing(cell, n_atoms, min_dist, seed, z_choices=(6,), z_lo=0.0) -> Specimen:
    """Random sequential addition: uniform positions, periodic in x,y, min spacing ``min_dist``.

    z is not periodic (the slab has an entrance and an exit face).  PCG64(seed).
    """
    cx, cy, cz = cell
    rng = np.random.Generator(np.random.PCG64(seed))
    nbx = max(1, int(cx // min_dist))
    nby = max(1, int(cy // min_dist))
    nbz = max(1, int(cz // min_dist))
    bx, by, bz = cx / nbx, cy / nby, cz / nbz
    buckets: dict = {}
    pts = np.empty((n_atoms, 3))
    count = 0
    tries = 0
    d2 = min_dist * min_dist
    batch = rng.random((4096, 3))
    bi = 0
    while count < n_atoms:
        if bi == len(batch):
            batch = rng.random((4096, 3))
            bi = 0
        p = batch[bi] * (cx, cy, cz)
        bi += 1
        tries += 1
        if tries > 200 * n_atoms:
            raise RuntimeError("random packing did not converge")
        ix, iy, iz = int(p[0] / bx) % nbx, int(p[1] / by) % nby, min(int(p[2] / bz), nbz - 1)
        ok = True
        for ddx in (-1, 0, 1):
            for ddy in (-1, 0, 1):
                for ddz in (-1, 0, 1):
                    kz = iz + ddz
                    if kz < 0 or kz >= nbz:
                        continue
                    for q in buckets.get(((ix + ddx) % nbx, (iy + ddy) % nby, kz), ()):
                        dx = p[0] - pts[q, 0]
                        dy = p[1] - pts[q, 1]
                        dx -= cx * round(dx / cx)
                        dy -= cy * round(dy / cy)
                        dzz = p[2] - pts[q, 2]
                        if dx * dx + dy * dy + dzz * dzz < d2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if not ok:
            continue
        pts[count] = p
        buckets.setdefault((ix, iy, iz), []).append(count)
        count += 1
    pts[:, 2] += z_lo
    zc = np.asarray(z_choices)
    z = zc[rng.integers(0, len(zc), size=n_atoms)] if len(zc) > 1 else np.full(n_atoms, zc[0])
    return Specimen(pts, z.astype(np.int64), (cx, cy, cz + z_lo),
                    note=f"random packing n={n_atoms} dmin={min_dist} seed={seed}")


def fcc_sphere_on_block(seed=3, block=(32.0, 32.0, 16.0), block_a=2.0, block_z=29,
                        particle_diameter=20.0, particle_a=4.08, particle_z=79) -> Specimen:
    """fcc sphere (seeded random rotation) resting on the entrance side of a simple-cubic block.

    The particle occupies z in [0, diameter); the block follows below it.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    cx, cy, cz = block
    n = int(round(cx / block_a)), int(round(cy / block_a)), int(round(cz / block_a))
    i, j, k = np.meshgrid(*(np.arange(m) for m in n), indexing="ij")
    blk = np.stack([i.ravel() * block_a, j.ravel() * block_a,
                    particle_diameter + (k.ravel() + 0.5) * block_a], axis=1)
    r = particle_diameter / 2
    m = int(math.ceil(r / particle_a)) + 1
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.stack(np.meshgrid(*(np.arange(-m, m + 1),) * 3, indexing="ij"), -1).reshape(-1, 3)
    lat = ((g[:, None, :] + basis[None]) * particle_a).reshape(-1, 3)
    lat = lat[np.einsum("ij,ij->i", lat, lat) <= r * r]
    qv = rng.normal(size=4)
    qv /= np.linalg.norm(qv)
    w, x, y, z = qv
    rot = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                    [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                    [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
    lat = lat @ rot.T + np.array([cx / 2, cy / 2, r])
    xyz = np.concatenate([lat, blk])
    zn = np.concatenate([np.full(len(lat), particle_z), np.full(len(blk), block_z)])
    return Specimen(xyz, zn.astype(np.int64), (cx, cy, particle_diameter + cz),
                    note=f"fcc Z={particle_z} sphere d={particle_diameter} seed={seed} on SC Z={block_z}")


# ------------------------------------------------------------- potentials
def project_potential(spec: Specimen, nx: int, ny: int, n_slices: int, dz: float,
                      v0=V0_VA, sigma=SIGMA_G, cutoff=CUTOFF_SIGMAS) -> np.ndarray:
    """Projected potential slices [n_slices][ny][nx] float32 (V*Angstrom).

    Atom a with z in [p dz, (p+1) dz) adds v0 * Z**0.7 * exp(-|r - r_a|^2 / (2 sigma^2))
    to slice p at every pixel within ``cutoff*sigma`` of one of its periodic images.
    Pixel (ix, iy) sits at (ix * cx/nx, iy * cy/ny).
    """
    cx, cy = spec.cell[0], spec.cell[1]
    px, py = cx / nx, cy / ny
    out = np.zeros((n_slices, ny, nx), dtype=np.float64)
    rc = cutoff * sigma
    hx = int(math.ceil(rc / px)) + 1
    hy = int(math.ceil(rc / py)) + 1
    offx = np.arange(-hx, hx + 1)
    offy = np.arange(-hy, hy + 1)
    inv2s2 = 1.0 / (2.0 * sigma * sigma)
    slice_idx = np.floor(spec.xyz[:, 2] / dz).astype(np.int64)
    for a in range(len(spec.xyz)):
        p = slice_idx[a]
        if p < 0 or p >= n_slices:
            continue
        x, y = spec.xyz[a, 0], spec.xyz[a, 1]
        amp = v0 * float(spec.z_number[a]) ** 0.7
        ix0 = int(math.floor(x / px))
        iy0 = int(math.floor(y / py))
        gx = (ix0 + offx) * px - x
        gy = (iy0 + offy) * py - y
        r2 = gy[:, None] ** 2 + gx[None, :] ** 2
        val = np.where(r2 <= rc * rc, amp * np.exp(-r2 * inv2s2), 0.0)
        iy = (iy0 + offy) % ny
        ix = (ix0 + offx) % nx
        np.add.at(out[p], (iy[:, None], ix[None, :]), val)
    return out.astype(np.float32)


# --------------------------------------------------------------- workloads
def workload_small(**over) -> Workload:
    """Simple-cubic Cu cell 16^3 A, 256^2 grid, 8 slices of 2 A, 300 kV, 20 mrad, f=4, 16x16 probes at 1 A."""
    w = Workload(name="sc-cu-16A-256px-8sl-f4", nx=256, ny=256, cell_x=16.0, cell_y=16.0,
                 n_slices=8, dz=2.0, kv=300.0, f=4, alpha_mrad=20.0,
                 scan_px=16, scan_py=16, scan_step=1.0,
                 specimen=simple_cubic(16.0, 2.0, 29))
    for k, v in over.items():
        setattr(w, k, v)
    return w


def workload_amorphous_carbon(**over) -> Workload:
    """a-C slab 50x50x100 A, 0.1 atoms/A^3 (25000 atoms, seed 1, dmin 1.4 A), 1024^2, 50 slices, f=8,
    200x200 probes at 0.25 A."""
    spec = over.pop("specimen", None)
    if spec is None:
        spec = random_packing((50.0, 50.0, 100.0), 25000, 1.4, seed=1, z_choices=(6,))
    w = Workload(name="a-C-50A-1024px-50sl-f8", nx=1024, ny=1024, cell_x=50.0, cell_y=50.0,
                 n_slices=50, dz=2.0, kv=300.0, f=8, alpha_mrad=20.0,
                 scan_px=200, scan_py=200, scan_step=0.25, specimen=spec)
    for k, v in over.items():
        setattr(w, k, v)
    return w


def workload_nanoparticle(f=4, **over) -> Workload:
    """20 A fcc Au sphere (seed 3) on a 32x32x16 A SC Cu block, 512^2 grid (0.0625 A), 18 slices."""
    w = Workload(name=f"au-np-on-cu-512px-18sl-f{f}", nx=512, ny=512, cell_x=32.0, cell_y=32.0,
                 n_slices=18, dz=2.0, kv=300.0, f=f, alpha_mrad=20.0,
                 scan_px=32, scan_py=32, scan_step=0.25,
                 specimen=fcc_sphere_on_block(seed=3))
    for k, v in over.items():
        setattr(w, k, v)
    return w


def workload_batch_cell(seed: int) -> Workload:
    """One cell of the batched workload of uneven cells.  PCG64(seed) draws the grid N from
    {256, 512, 1024} (0.0625 A pixels, so the cell is N/16 A square), the slice count H from
    [10, 60] (2 A slices), f from {4, 8}; atoms by random sequential addition at 0.1 atoms/A^3 with
    1.4 A minimum spacing, each atom's Z drawn from {6, 14, 29, 79}.  Scan: 16 x 16 probes at
    0.25 A.  300 kV, 20 mrad."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = (256, 512, 1024)[int(rng.integers(0, 3))]
    h = int(rng.integers(10, 61))
    f = (4, 8)[int(rng.integers(0, 2))]
    cell = n * 0.0625
    n_atoms = int(round(0.1 * cell * cell * 2.0 * h))
    spec = random_packing((cell, cell, 2.0 * h), n_atoms, 1.4, seed=seed, z_choices=(6, 14, 29, 79))
    return Workload(name=f"batch-cell-{seed}-{n}px-{h}sl-f{f}", nx=n, ny=n, cell_x=cell, cell_y=cell,
                    n_slices=h, dz=2.0, kv=300.0, f=f, alpha_mrad=20.0,
                    scan_px=16, scan_py=16, scan_step=0.25, specimen=spec)


def batch_cell_potential(seed: int):
    """(workload, potential) of one batched cell; a top-level function so that process pools can map it."""
    w = workload_batch_cell(seed)
    return w, w.potential()


def potential_stats(v: np.ndarray) -> dict:
    return {"min": float(v.min()), "max": float(v.max()), "mean": float(v.mean())}


def displaced(spec: Specimen, u_rms: float, seed: int) -> Specimen:
    """One frozen-phonon configuration: every atom moved by an independent Gaussian displacement of
    standard deviation ``u_rms`` (Angstrom) along x, y and z.  PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xyz = spec.xyz + rng.normal(scale=u_rms, size=spec.xyz.shape)
    return Specimen(xyz, spec.z_number.copy(), spec.cell, note=spec.note + f" displaced u_rms={u_rms} seed={seed}")
