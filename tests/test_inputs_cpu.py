"""The seeded synthetic inputs: the specimens and scans the workloads are built from keep the
properties their recipes state (atom counts and densities, minimum spacing under the periodic x, y
boundary, cell sizes, scan rasters, seed reproducibility).  CPU only."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from paper_1702_01904_gb300 import specimens as S


def min_spacing(spec):
    # periodic in x and y, open along z (a z period far beyond the slab never wraps)
    cx, cy, cz = spec.cell
    tree = cKDTree(np.mod(spec.xyz, (cx, cy, 4 * cz + 1.0)), boxsize=(cx, cy, 4 * cz + 1.0))
    d, _ = tree.query(np.mod(spec.xyz, (cx, cy, 4 * cz + 1.0)), k=2)
    return d[:, 1].min()


def test_random_packing_spacing_density_and_seed():
    a = S.random_packing((20.0, 20.0, 20.0), 800, 1.4, seed=5, z_choices=(6, 14, 29, 79))
    assert a.xyz.shape == (800, 3)
    assert np.all(a.xyz >= 0) and np.all(a.xyz < (20.0, 20.0, 20.0))
    assert min_spacing(a) >= 1.4
    assert set(np.unique(a.z_number)) <= {6, 14, 29, 79}
    b = S.random_packing((20.0, 20.0, 20.0), 800, 1.4, seed=5, z_choices=(6, 14, 29, 79))
    c = S.random_packing((20.0, 20.0, 20.0), 800, 1.4, seed=6, z_choices=(6, 14, 29, 79))
    assert np.array_equal(a.xyz, b.xyz) and np.array_equal(a.z_number, b.z_number)
    assert not np.array_equal(a.xyz, c.xyz)


def test_amorphous_carbon_workload_recipe():
    w = S.workload_amorphous_carbon()
    s = w.specimen
    assert s.xyz.shape == (25000, 3) and np.all(s.z_number == 6)
    assert s.cell == (50.0, 50.0, 100.0)
    assert abs(len(s.xyz) / (50.0 * 50.0 * 100.0) - 0.1) < 1e-12
    assert min_spacing(s) >= 1.4
    assert (w.nx, w.ny, w.n_slices, w.dz, w.f, w.kv, w.alpha_mrad) == (1024, 1024, 50, 2.0, 8, 300.0, 20.0)
    # every atom falls in one of the 50 slices of 2 A
    assert s.xyz[:, 2].max() < w.n_slices * w.dz
    x0, y0 = w.scan_positions()
    assert len(x0) == 40000 and x0[1] - x0[0] == 0.25 and y0[200] - y0[0] == 0.25
    assert x0.max() == 199 * 0.25 and y0.max() == 199 * 0.25


@pytest.mark.parametrize("seed", [101, 104])
def test_batch_cell_recipe(seed):
    w = S.workload_batch_cell(seed)
    assert w.nx in (256, 512, 1024) and w.ny == w.nx and w.cell_x == w.nx * 0.0625
    assert 10 <= w.n_slices <= 60 and w.f in (4, 8) and w.dz == 2.0
    s = w.specimen
    assert len(s.xyz) == round(0.1 * w.cell_x * w.cell_y * 2.0 * w.n_slices)
    assert min_spacing(s) >= 1.4
    assert set(np.unique(s.z_number)) <= {6, 14, 29, 79}
    assert (w.scan_px, w.scan_py, w.scan_step) == (16, 16, 0.25)
    assert S.workload_batch_cell(seed).name == w.name


def test_displaced_configuration_statistics():
    spec = S.random_packing((30.0, 30.0, 20.0), 1800, 1.4, seed=7)
    d = S.displaced(spec, 0.1, seed=11)
    u = d.xyz - spec.xyz
    assert u.shape == spec.xyz.shape and np.array_equal(d.z_number, spec.z_number)
    # 5400 independent N(0, 0.1^2) draws: the sample rms is 0.1 within a few per cent
    assert abs(np.sqrt((u ** 2).mean()) - 0.1) < 0.005 and abs(u.mean()) < 0.005
    assert np.array_equal(S.displaced(spec, 0.1, seed=11).xyz, d.xyz)


def test_projected_potential_slices_partition_the_atoms():
    # a single atom contributes to exactly the slice that holds its z, with the Gaussian's peak
    spec = S.Specimen(np.array([[4.0, 4.0, 3.0]]), np.array([29]), (8.0, 8.0, 8.0))
    v = S.project_potential(spec, 64, 64, 4, 2.0)
    assert np.count_nonzero(v.reshape(4, -1).max(1) > 0) == 1 and v[1].max() > 0
    assert abs(v.max() - S.V0_VA * 29 ** 0.7) / (S.V0_VA * 29 ** 0.7) < 1e-3


def test_chunked_packing_spacing_density_and_seed():
    a = S.random_packing_chunked((30.0, 30.0, 24.0), 2160, 1.4, seed=8, chunk=256)
    assert a.xyz.shape == (2160, 3)
    assert np.all(a.xyz >= 0) and np.all(a.xyz < (30.0, 30.0, 24.0))
    assert min_spacing(a) >= 1.4
    assert np.array_equal(S.random_packing_chunked((30.0, 30.0, 24.0), 2160, 1.4, seed=8, chunk=256).xyz, a.xyz)
    # positions are uniform: each half of the cell along every axis holds about half the atoms
    for ax, c in enumerate((30.0, 30.0, 24.0)):
        assert abs(np.mean(a.xyz[:, ax] < c / 2) - 0.5) < 0.05


def test_large_serving_cell_recipe():
    # a thin version of the 2048^2 cell: the Au sphere on the entrance side, carbon below it
    w = S.workload_nanoparticle_on_carbon(n_slices=8, particle_diameter=10.0)
    s = w.specimen
    assert (w.nx, w.ny, w.cell_x, w.f, w.n_slices, w.dz) == (2048, 2048, 102.4, 8, 8, 2.0)
    au, c = s.xyz[s.z_number == 79], s.xyz[s.z_number == 6]
    assert len(au) > 20 and np.all(au[:, 2] < 10.0 + 1e-9)
    assert np.all(np.abs(au[:, :2] - 51.2).max(1) <= 5.0 + 1e-9)
    assert abs(len(c) - 0.1 * 102.4 * 102.4 * 6.0) < 1 and np.all(c[:, 2] >= 10.0) and np.all(c[:, 2] < 16.0)
    assert min_spacing(S.Specimen(c, s.z_number[s.z_number == 6], (102.4, 102.4, 16.0))) >= 1.4
    # the full-thickness recipe: 40 A sphere over 160 A of carbon (about 168 000 carbon atoms)
    assert round(0.1 * 102.4 * 102.4 * (200.0 - 40.0)) == 167772


def test_vectorised_projection_equals_the_per_atom_one():
    spec = S.nanoparticle_on_carbon(16.0, 8.0, 4.0, seed=9)
    ref = S.project_potential(spec, 128, 128, 4, 2.0)
    got = S.project_potential_vectorised(spec, 128, 128, 4, 2.0, chunk=37)
    assert np.max(np.abs(got - ref)) <= 1e-6 * np.max(ref)
