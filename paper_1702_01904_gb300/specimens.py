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


def random_packing_chunked(cell, n_atoms, min_dist, seed, z_choices=(6,), z_lo=0.0, chunk=1024) -> Specimen:
    """Random sequential addition for cells of 10^5 atoms and more, vectorised over chunks of
    candidates.  Candidates are uniform in the cell (PCG64(seed)) and are taken in draw order; one is
    kept when it lies at least ``min_dist`` from every atom kept before it (periodic in x, y; z is not
    periodic), which is the same acceptance rule as ``random_packing`` evaluated with NumPy arrays
    (a bucket grid of side >= min_dist holds the kept atoms).  The draws differ from
    ``random_packing``, so the atoms differ for the same seed."""
    cx, cy, cz = cell
    rng = np.random.Generator(np.random.PCG64(seed))
    nbx, nby, nbz = max(3, int(cx // min_dist)), max(3, int(cy // min_dist)), max(1, int(cz // min_dist))
    bx, by, bz = cx / nbx, cy / nby, cz / nbz
    cap = 16  # atoms at >= min_dist apart in one bucket of side < 2 min_dist: at most 8 (corners)
    occ = np.full((nbx, nby, nbz, cap), -1, dtype=np.int64)
    fill = np.zeros((nbx, nby, nbz), dtype=np.int64)
    pts = np.empty((n_atoms, 3))
    count = 0
    d2 = min_dist * min_dist
    offs = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)])
    draws = 0
    while count < n_atoms:
        draws += chunk
        if draws > 200 * n_atoms + chunk:
            raise RuntimeError("random packing did not converge")
        cand = rng.random((chunk, 3)) * (cx, cy, cz)
        ix = (cand[:, 0] / bx).astype(np.int64) % nbx
        iy = (cand[:, 1] / by).astype(np.int64) % nby
        iz = np.minimum((cand[:, 2] / bz).astype(np.int64), nbz - 1)
        # conflicts with atoms kept in earlier chunks: the 27 neighbouring buckets
        nx_ = (ix[:, None] + offs[None, :, 0]) % nbx
        ny_ = (iy[:, None] + offs[None, :, 1]) % nby
        nz_ = iz[:, None] + offs[None, :, 2]
        zin = (nz_ >= 0) & (nz_ < nbz)
        idx = occ[nx_, ny_, np.clip(nz_, 0, nbz - 1)]          # [chunk, 27, cap]
        idx = np.where(zin[:, :, None], idx, -1).reshape(chunk, -1)
        valid = idx >= 0
        q = pts[np.where(valid, idx, 0)]
        dx = cand[:, None, 0] - q[:, :, 0]
        dy = cand[:, None, 1] - q[:, :, 1]
        dx -= cx * np.round(dx / cx)
        dy -= cy * np.round(dy / cy)
        dzz = cand[:, None, 2] - q[:, :, 2]
        clash = np.any(valid & (dx * dx + dy * dy + dzz * dzz < d2), axis=1)
        surv = np.flatnonzero(~clash)
        # conflicts inside the chunk: a candidate is dropped if an earlier kept one is too close
        sc = cand[surv]
        ddx = sc[:, None, 0] - sc[None, :, 0]
        ddy = sc[:, None, 1] - sc[None, :, 1]
        ddx -= cx * np.round(ddx / cx)
        ddy -= cy * np.round(ddy / cy)
        ddz = sc[:, None, 2] - sc[None, :, 2]
        near = np.triu(ddx * ddx + ddy * ddy + ddz * ddz < d2, k=1)
        keep = np.ones(len(surv), dtype=bool)
        for i, j in zip(*np.nonzero(near)):
            if keep[i]:
                keep[j] = False
        for k in surv[keep]:
            if count == n_atoms:
                break
            b = (ix[k], iy[k], iz[k])
            if fill[b] == cap:
                raise RuntimeError("random packing bucket overflow")
            occ[b + (fill[b],)] = count
            fill[b] += 1
            pts[count] = cand[k]
            count += 1
    pts[:, 2] += z_lo
    zc = np.asarray(z_choices)
    z = zc[rng.integers(0, len(zc), size=n_atoms)] if len(zc) > 1 else np.full(n_atoms, zc[0])
    return Specimen(pts, z.astype(np.int64), (cx, cy, cz + z_lo),
                    note=f"random packing (chunked) n={n_atoms} dmin={min_dist} seed={seed}")


def fcc_sphere(diameter, a, z_number, seed, centre) -> Specimen:
    """fcc sphere of the given diameter, lattice constant ``a`` and seeded random rotation
    (PCG64(seed) quaternion), centred at ``centre`` (x, y, z)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = diameter / 2
    m = int(math.ceil(r / a)) + 1
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.stack(np.meshgrid(*(np.arange(-m, m + 1),) * 3, indexing="ij"), -1).reshape(-1, 3)
    lat = ((g[:, None, :] + basis[None]) * a).reshape(-1, 3)
    lat = lat[np.einsum("ij,ij->i", lat, lat) <= r * r]
    qv = rng.normal(size=4)
    qv /= np.linalg.norm(qv)
    w, x, y, z = qv
    rot = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                    [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                    [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
    xyz = lat @ rot.T + np.asarray(centre, dtype=np.float64)
    return Specimen(xyz, np.full(len(xyz), z_number, dtype=np.int64), (diameter,) * 3,
                    note=f"fcc Z={z_number} sphere d={diameter} seed={seed}")


def nanoparticle_on_carbon(cell_xy=102.4, thickness=200.0, particle_diameter=40.0, seed=5) -> Specimen:
    """An fcc Au sphere (a = 4.08 A, seeded rotation) centred in x, y on the entrance side
    (z in [0, d)), above an amorphous-carbon support filling z in [d, thickness) at 0.1 atoms/A^3
    with 1.4 A minimum spacing (chunked random sequential addition, PCG64(seed + 1))."""
    d = particle_diameter
    au = fcc_sphere(d, 4.08, 79, seed, (cell_xy / 2, cell_xy / 2, d / 2)) if d > 0 else None
    parts = [] if au is None else [au]
    depth = thickness - d
    if depth > 0:
        n_c = int(round(0.1 * cell_xy * cell_xy * depth))
        parts.append(random_packing_chunked((cell_xy, cell_xy, depth), n_c, 1.4, seed + 1, (6,), z_lo=d))
    xyz = np.concatenate([p.xyz for p in parts])
    zn = np.concatenate([p.z_number for p in parts])
    return Specimen(xyz, zn, (cell_xy, cell_xy, thickness),
                    note=f"Au fcc sphere d={d} (seed {seed}) on a-C {depth:g} A thick (seed {seed + 1})")


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


def project_potential_vectorised(spec: Specimen, nx: int, ny: int, n_slices: int, dz: float,
                                 v0=V0_VA, sigma=SIGMA_G, cutoff=CUTOFF_SIGMAS, chunk=512) -> np.ndarray:
    """The same projected potential as ``project_potential`` (the same Gaussians, cutoff, slice
    assignment and pixel positions), evaluated for chunks of atoms at once: each stamp is the outer
    product of the Gaussian's x and y factors, and each chunk's stamps are summed with one
    ``np.bincount``.  The values agree with ``project_potential`` to FP64 rounding (the factored
    exponential and the order of the additions differ).  For cells of 10^5 atoms."""
    cx, cy = spec.cell[0], spec.cell[1]
    px, py = cx / nx, cy / ny
    rc = cutoff * sigma
    hx = int(math.ceil(rc / px)) + 1
    hy = int(math.ceil(rc / py)) + 1
    offx = np.arange(-hx, hx + 1)
    offy = np.arange(-hy, hy + 1)
    inv2s2 = 1.0 / (2.0 * sigma * sigma)
    slice_idx = np.floor(spec.xyz[:, 2] / dz).astype(np.int64)
    amp_all = v0 * spec.z_number.astype(np.float64) ** 0.7
    out = np.zeros((n_slices, ny, nx), dtype=np.float32)
    for p in range(n_slices):
        sel = np.flatnonzero(slice_idx == p)
        acc = np.zeros(nx * ny, dtype=np.float64)
        for c0 in range(0, len(sel), chunk):
            a = sel[c0:c0 + chunk]
            x, y = spec.xyz[a, 0], spec.xyz[a, 1]
            ix0 = np.floor(x / px).astype(np.int64)
            iy0 = np.floor(y / py).astype(np.int64)
            gx = (ix0[:, None] + offx[None, :]) * px - x[:, None]
            gy = (iy0[:, None] + offy[None, :]) * py - y[:, None]
            gx2, gy2 = gx * gx, gy * gy
            ex = np.exp(-gx2 * inv2s2)
            ey = amp_all[a][:, None] * np.exp(-gy2 * inv2s2)
            val = ey[:, :, None] * ex[:, None, :]
            val[gy2[:, :, None] + gx2[:, None, :] > rc * rc] = 0.0
            flat = ((iy0[:, None] + offy[None, :]) % ny)[:, :, None] * nx + ((ix0[:, None] + offx[None, :]) % nx)[:, None, :]
            acc += np.bincount(flat.ravel(), weights=val.ravel(), minlength=nx * ny)
        out[p] = acc.reshape(ny, nx)
    return out


def _project_slices(args):
    spec, nx, ny, p0, p1, dz = args
    sub = np.flatnonzero((spec.xyz[:, 2] >= p0 * dz) & (spec.xyz[:, 2] < p1 * dz))
    part = Specimen(spec.xyz[sub] - np.array([0.0, 0.0, p0 * dz]), spec.z_number[sub], spec.cell)
    return project_potential_vectorised(part, nx, ny, p1 - p0, dz)


def project_potential_parallel(spec: Specimen, nx: int, ny: int, n_slices: int, dz: float, workers=None) -> np.ndarray:
    """``project_potential_vectorised`` split over groups of slices in a pool of spawned processes
    (each slice depends only on its own atoms, so the result is the same array)."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor

    workers = workers or min(16, os.cpu_count() or 1)
    step = max(1, -(-n_slices // (2 * workers)))
    jobs = [(spec, nx, ny, p0, min(n_slices, p0 + step), dz) for p0 in range(0, n_slices, step)]
    out = np.empty((n_slices, ny, nx), dtype=np.float32)
    with ProcessPoolExecutor(min(workers, len(jobs)), mp_context=mp.get_context("spawn")) as ex:
        for (_, _, _, p0, p1, _), v in zip(jobs, ex.map(_project_slices, jobs)):
            out[p0:p1] = v
    return out


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


def workload_nanoparticle_on_carbon(n_slices=100, particle_diameter=40.0, seed=5, **over) -> Workload:
    """Large serving cell: 102.4 x 102.4 A, 2048^2 grid (0.05 A pixels), ``n_slices`` slices of 2 A,
    300 kV, 20 mrad, f = 8 (529 beams).  Specimen: ``nanoparticle_on_carbon`` with the cell's
    thickness (40 A Au sphere on 160 A of a-C at 100 slices, about 170 000 atoms).  Default scan: a
    64 x 64 region of interest at 0.25 A."""
    spec = over.pop("specimen", None)
    if spec is None:
        spec = nanoparticle_on_carbon(102.4, 2.0 * n_slices, particle_diameter, seed)
    w = Workload(name=f"au-np-on-aC-2048px-{n_slices}sl-f8", nx=2048, ny=2048, cell_x=102.4, cell_y=102.4,
                 n_slices=n_slices, dz=2.0, kv=300.0, f=8, alpha_mrad=20.0,
                 scan_px=64, scan_py=64, scan_step=0.25, specimen=spec)
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
