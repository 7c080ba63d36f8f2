"""The seeded workload recipes (paper_2506_04763_gb300/inputs.py) against the
recipe they state: fluids and materials, the hydrostatic initial state with its
NAPL blob, the lognormal field's moments and correlation length, the lenses,
the DNAPL inlet, the ensemble's seeds and sizes, and the Buckley-Leverett
strip's boundary data.  CPU only."""
import numpy as np
import pytest

from paper_2506_04763_gb300 import inputs as I


def _cells3(p):
    n = p["n"]
    return (n[2] - 1, n[1] - 1, n[0] - 1)


def test_fluids_materials_and_grid():
    p = I.lens_square_2d()
    assert (p["rho_w"], p["rho_n"], p["mu_w"], p["mu_n"]) == (1000.0, 1460.0, 1e-3, 9e-4)
    assert (p["S_wr"], p["S_nr"], p["lam"]) == (0.10, 0.0, 2.0)
    assert p["n"] == (33, 33, 1) and p["h"][:2] == (1.0 / 32, 1.0 / 32)
    assert p["g"] == (0.0, -9.81, 0.0)
    # the centred 9x5-cell lens: x-cells [11, 20), y-cells [13, 18)
    pd = p["pd"].reshape(32, 32)
    lens = np.zeros((32, 32), bool)
    lens[13:18, 11:20] = True
    assert np.all(pd[lens] == 1163.0) and np.all(pd[~lens] == 755.0)
    assert np.all(p["K"].reshape(32, 32)[lens] == 3.32e-11) and np.all(p["phi"].reshape(32, 32)[lens] == 0.39)
    assert np.all(p["K"].reshape(32, 32)[~lens] == 6.64e-11) and np.all(p["phi"].reshape(32, 32)[~lens] == 0.40)


@pytest.mark.parametrize("dim,nv", [(2, (33, 33)), (3, (17, 17, 17))])
def test_initial_state_is_hydrostatic_with_a_clipped_blob(dim, nv):
    n, h, _ = I.grid(dim, nv)
    u = I.initial_state(dim, n, h, seed=0)
    x, y, z = I._coords(dim, n, h)
    vert = y if dim == 2 else z
    top = I.top_mask(dim, n).astype(bool)
    pw, sn = u[0::2], u[1::2]
    assert np.all(pw[top] == 1e5)
    noise = pw[~top] - (1e5 + 1000.0 * 9.81 * (1.0 - vert[~top]))
    assert abs(noise.mean()) < 1.0 and 8.0 < noise.std() < 12.0          # N(0, 10 Pa)
    assert sn.min() >= 0.0 and sn.max() <= 0.8
    r2 = (x - 0.5) ** 2 + ((y - 1.0) ** 2 if dim == 2 else (y - 0.5) ** 2 + (z - 1.0) ** 2)
    np.testing.assert_allclose(sn, np.clip(0.3 * np.exp(-r2 / 0.05), 0.0, 0.8), rtol=0, atol=0)


def test_lognormal_field_moments_and_correlation_length():
    """ln K = ln 5e-11 + f, f standardised exactly; its correlation at lag r
    cells follows exp(-r^2 / l^2) with l = 8 (sampled along all three axes)."""
    n = (65, 65, 65)
    K, _ = I.lognormal_field(3, n, seed=1)
    lk = np.log(K)
    assert lk.mean() == pytest.approx(np.log(5e-11), abs=1e-9)
    assert lk.std() == pytest.approx(1.0, rel=1e-9)
    f = (lk - lk.mean()).reshape(64, 64, 64)
    for r in (2, 4, 8):
        c = np.mean([np.mean(np.roll(f, r, axis=a) * f) for a in range(3)]) / f.var()
        assert c == pytest.approx(np.exp(-r * r / 64.0), abs=0.12), (r, c)


def test_lenses_are_boxes_of_the_stated_extent_and_values():
    p = I.lognormal_lenses_box(65)
    q = I.lognormal_box(65, seed=2)        # the same field without lenses
    lens = (p["pd"] == 1163.0).reshape(_cells3(p))
    assert lens.any() and np.all(p["pd"][~lens.ravel()] == 755.0)
    # inside a lens K is the field's K / 20, once per lens covering the cell
    # (overlapping lenses multiply); outside the field is untouched
    ratio = (p["K"] / q["K"]).reshape(_cells3(p))
    assert np.all(ratio[~lens] == 1.0)
    k = np.log(ratio[lens]) / np.log(1.0 / 20.0)
    assert np.all(np.abs(k - np.rint(k)) < 1e-9) and k.min() > 0.5 and np.any(np.rint(k) == 1)
    # lens extents are drawn from U[8, 32] cells: the lenses cover at least 8
    # cells along every axis
    for ax in range(3):
        cover = lens.any(axis=tuple(b for b in range(3) if b != ax))
        assert cover.sum() >= 8
    assert np.array_equal(p["phi"], q["phi"])


def test_dnapl_inlet_and_boundary_masks():
    nv = 33
    p = I.dnapl_infiltration(nv)
    n, h = p["n"], p["h"]
    x, y, z = I._coords(3, n, h)
    top = z == 1.0
    q = p["q_in"]
    assert np.all(q[0::2] == 0.0)
    inlet = q[1::2] > 0.0
    assert np.all(top[inlet]) and np.all(np.abs(x[inlet] - 0.5) <= 0.05 + 1e-12)
    assert np.all(np.abs(y[inlet] - 0.5) <= 0.05 + 1e-12)
    # each inlet vertex (interior of the top face) takes 0.1 kg m^-2 s^-1 over
    # its dual face h_x h_y; the patch is the vertices within 0.05 of the centre
    assert np.allclose(q[1::2][inlet], 0.1 * h[0] * h[1], rtol=1e-14, atol=0)
    m = int(np.sum(np.abs(np.arange(n[0]) * h[0] - 0.5) <= 0.05 + 1e-12))
    assert inlet.sum() == m * m
    dm = p["dir"].astype(bool)
    assert np.array_equal(dm, top & ~inlet)
    assert np.all(p["pw_dir"][dm] == 1e5) and np.all(p["pw_dir"][~dm] == 0.0)


def test_ensemble_seeds_and_sizes():
    m = I.ensemble_members()
    assert [s for s, _ in m] == list(range(100, 164))
    assert [v for _, v in m] == [33] * 16 + [49] * 16 + [65] * 16 + [97] * 16
    p = I.ensemble_member(100, 33)
    assert p["n"] == (33, 33, 33) and p["nlevels"] == 4 and np.all(p["pd"] == 755.0)
    assert I.levels_for(257) == 7 and I.levels_for(385) == 8 and I.levels_for(97) == 6


def test_buckley_leverett_strip_boundary_data():
    c = I.CASE1
    p = I.case1_buckley_leverett(64)
    nx, ny = 64, 9
    assert p["n"] == (nx + 1, ny, 1) and p["h"][0] == pytest.approx(c["L"] / nx)
    i = np.arange((nx + 1) * ny) % (nx + 1)
    # water-filled inlet column held at p_in; NAPL everywhere else
    assert np.array_equal(p["dir"].astype(bool), i == 0)
    assert np.all(p["u0"][1::2][i == 0] == 0.0) and np.all(p["u0"][1::2][i > 0] == 1.0)
    # the outlet sink removes q_out per unit outlet length (the strip's 75 m)
    assert p["q_in"][1::2].sum() == pytest.approx(-c["q_out"] * c["W"], rel=1e-12)
    assert np.all(p["q_in"][1::2][i < nx] == 0.0)
