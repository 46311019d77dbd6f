"""The seeded synthetic inputs (workloads.py) have the configurations' sizes, coarse spaces,
boundary conditions and structure, and are reproducible."""
import numpy as np
import pytest

import workloads

# (nelx, nely, DOFs, coarse nodes N_c, coarse unknowns N_t) of the five configurations
SIZES = {
    "mbb_c1": (192, 64, 25_090, 65, 260),
    "mbb_c2": (1024, 512, 1_051_650, 561, 3_366),
    "mbb_c3": (2048, 1024, 4_200_450, 2_145, 12_870),
    "mbb_c5": (3200, 4096, 26_228_994, 13_029, 78_174),
}


@pytest.mark.parametrize("name", sorted(SIZES))
def test_configuration_sizes_and_coarse_spaces(name):
    wl = workloads.make(name)
    nelx, nely, dofs, nc, nt = SIZES[name]
    assert (wl.nelx, wl.nely) == (nelx, nely)
    assert 2 * (wl.nelx + 1) * (wl.nely + 1) == dofs
    assert wl.nelx % wl.H == 0 and wl.nely % wl.H == 0
    assert (wl.nelx // wl.H + 1) * (wl.nely // wl.H + 1) == nc
    assert nc * wl.n_eig == nt


@pytest.mark.parametrize("name", ["mbb_c1", "mbb_c2", "mbb_c3"])
def test_mbb_boundary_conditions(name):
    """MBB half beam: u_x = 0 on the left edge, u_y = 0 at the bottom-right node, one unit
    downward load at the top-left node (nodal layout [nely+1][nelx+1][2])."""
    wl = workloads.make(name, 4)
    fixed = np.asarray(wl.fixed).reshape(wl.nely + 1, wl.nelx + 1, 2)
    force = np.asarray(wl.force).reshape(wl.nely + 1, wl.nelx + 1, 2)
    assert fixed[:, 0, 0].all() and fixed.sum() == (wl.nely + 1) + 1
    assert fixed[0, wl.nelx, 1]
    assert np.count_nonzero(force) == 1 and force[wl.nely, 0, 1] == -1.0


def test_workloads_are_reproducible():
    for name in ("mbb_c1", "mbb_c3"):
        a, b = workloads.make(name, 4), workloads.make(name, 4)
        assert np.array_equal(a.rho, b.rho)
    ba, bb = workloads.cantilever_batch(8, scale=4), workloads.cantilever_batch(8, scale=4)
    assert [(w.nelx, w.nely) for w in ba] == [(w.nelx, w.nely) for w in bb]
    assert all(np.array_equal(x.rho, y.rho) for x, y in zip(ba, bb))


def test_structures():
    """C2: a Bernoulli(0.4) void cell; C5: a radius-10 void in a 32x32 cell (area pi r^2);
    C3: alternating layers of thickness 4..12, every void layer crossed by 8-wide struts
    every 32 elements."""
    c2 = workloads.make("mbb_c2")
    assert c2.rho.shape == (32, 32) and abs((c2.rho == 0).mean() - 0.4) < 0.06
    c5 = workloads.make("mbb_c5")
    assert c5.rho.shape == (32, 32)
    assert abs((1.0 - c5.rho).sum() - np.pi * 100.0) < 20.0
    c3 = workloads.make("mbb_c3", 4)
    rows_full = (c3.rho == 1.0).all(axis=1)
    frac = c3.rho.mean(axis=1)
    assert np.all(rows_full | np.isclose(frac, 8.0 / 32.0, atol=1.0 / c3.nelx + 1e-12))
    # layer thicknesses: runs of equal row type
    kinds = rows_full.astype(int)
    edges = np.flatnonzero(np.diff(kinds)) + 1
    runs = np.diff(np.r_[0, edges, len(kinds)])
    assert runs[:-1].min() >= 4 and runs.max() <= 12


def test_uneven_batch():
    """C4: 64 cantilevers of the five sizes, 26,178,048 DOFs in all, H 16, k 4."""
    batch = workloads.cantilever_batch()
    assert len(batch) == 64
    sizes = {(w.nelx, w.nely) for w in batch}
    assert sizes <= {(256, 128), (384, 192), (512, 256), (768, 384), (1024, 512)}
    assert sum(2 * (w.nelx + 1) * (w.nely + 1) for w in batch) == 26_178_048
    assert all(w.H == 16 and w.n_eig == 4 for w in batch)


def test_literal_layers_are_the_strut_layers_without_struts():
    """mbb_c3_literal: the same seeded layer sequence as mbb_c3 with every void layer fully
    void (no struts), so the stiff layers do not touch one another."""
    lit, st = workloads.make("mbb_c3_literal", 4), workloads.make("mbb_c3", 4)
    assert lit.rho.shape == st.rho.shape and (lit.rho <= st.rho).all()
    rows_lit, rows_st = lit.rho.max(axis=1), st.rho.min(axis=1)
    assert set(np.unique(lit.rho)) <= {0.0, 1.0}
    # a row is solid in both or void in the literal layers (struts only fill void rows)
    assert np.array_equal(rows_lit == 1.0, rows_st == 1.0)
    assert (lit.rho[rows_lit == 0.0] == 0.0).all() and (st.rho[rows_lit == 0.0] > 0.0).any()
