"""GPU parity of gridff_langevin (BAOAB with the counter-based noise stream)
and of the flexible RMSD uniqueness filter against the oracle, plus the
thermostat's temperature."""
import numpy as np
import pytest

from oracle import dynamics as odyn
from oracle import grid as ogrid
from oracle import sampling as osamp
from paper_2508_15522_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import __graft_entry__ as ge
    ge.build()
    from paper_2508_15522_gb300 import gridff
    return gridff


@pytest.fixture(scope="module")
def ctx(G):
    return G.Context(0)


@pytest.fixture(scope="module")
def field(G, ctx):
    sub = synth.rocksalt_slab(ncell=2)
    box = synth.grid_box_for(sub, 0.25, height=8.0)
    n, h = ogrid.grid_dims(box.length, box.spacing)
    coefs = synth.random_coefficients(n, 3, seed=151, scale=(0.02, 0.01, 0.03))
    grid = G.grid_from_coefs(ctx, coefs, box.origin, h, 7)
    return sub, box, h, coefs.astype(np.float32).astype(np.float64), grid


@pytest.mark.parametrize("wpb", [2, 8])
def test_langevin_steps_match_oracle(G, ctx, field, wpb):
    sub, box, h, c32, grid = field
    mol = synth.chain_molecule()
    n_rep, seed, dt, T, gamma = 11, 0xABCDEF, 0.5, 300.0, 0.05
    x0 = synth.flexible_positions(mol, sub, n_rep, seed=152).astype(np.float32)
    v0 = (0.003 * synth.rng(153).standard_normal(x0.shape)).astype(np.float32)
    fn = odyn.make_force_fn(c32, ("C", "P", "L"), box.origin, h, mol)
    reps = G.Replicas(ctx, [mol], [0] * n_rep)
    reps.set_launch_config(kernel=G.KERNEL_FLEX_TERMS, warps_per_block=wpb, cache_slots=0, queue=1)
    reps.set_state(x0.ravel(), v0.ravel())
    # two calls (steps 0-3, then 4-9) continue one noise stream
    G.langevin(ctx, grid, reps, 4, dt, T, gamma, seed, step0=0)
    G.langevin(ctx, grid, reps, 6, dt, T, gamma, seed, step0=4)
    x, v = reps.get_state()
    noise = lambda s: odyn.langevin_noise(seed, range(n_rep), s, 3 * mol.n)
    xr, vr, Er = odyn.langevin_baoab(x0.astype(np.float64), v0.astype(np.float64), mol.mass, fn, 10, dt, T, gamma,
                                     noise)
    assert np.abs(x.reshape(xr.shape) - xr).max() < 5e-5
    assert np.abs(v.reshape(vr.shape) - vr).max() < 5e-5
    assert np.allclose(reps.fire_state()["energy"], Er, atol=1e-4 * mol.n)
    reps.close()


def test_langevin_thermostat_temperature(G, ctx, field):
    """Equipartition: after thermalisation the kinetic temperature of many
    replicas is T (3n degrees of freedom each)."""
    sub, box, h, c32, grid = field
    mol = synth.random_flexible_molecule(24, 4, 154)
    n_rep, T = 512, 300.0
    x0 = synth.flexible_positions(mol, sub, n_rep, seed=155, h_lo=3.5, h_hi=4.5).astype(np.float32)
    reps = G.Replicas(ctx, [mol], [0] * n_rep)
    reps.set_state(x0.ravel())
    G.langevin(ctx, grid, reps, 3000, 0.5, T, 0.02, 7)
    temps = []
    for k in range(5):
        G.langevin(ctx, grid, reps, 200, 0.5, T, 0.02, 7, step0=3000 + 200 * k)
        x, v = reps.get_state()
        ke = 0.5 * np.sum(np.tile(mol.mass, n_rep)[:, None] * v.reshape(-1, 3) ** 2) / odyn.ACC
        temps.append(2 * ke / (3 * mol.n * n_rep * odyn.KB))
    assert abs(np.mean(temps) / T - 1) < 0.03, temps


def test_rmsd_unique_xyz_matches_oracle(G, ctx):
    g = synth.rng(156)
    mol = synth.random_flexible_molecule(20, 3, 157)
    tile = (11.28, 11.28)
    base = [mol.xyz + [g.uniform(0, 11), g.uniform(0, 11), 6.0] for _ in range(40)]
    near = [b + g.normal(0, 0.01, b.shape) for b in base]
    far = [b + g.normal(0, 0.3, b.shape) for b in base]
    img = [b + [tile[0] * g.integers(-2, 3), -tile[1], 0.0] for b in base]
    S = np.array(base + near + far + img)
    S = S[g.permutation(len(S))].astype(np.float32)
    ref = osamp.dup_of_xyz(S.astype(np.float64), tile, 0.1)
    for i in range(len(S)):
        for j in range(i):
            assert abs(osamp.rmsd_xyz(S[i], S[j], tile) - 0.1) > 0.01
    got = G.rmsd_unique_xyz(ctx, S, tile, 0.1)
    assert got.tolist() == ref.tolist()
    assert 80 <= np.sum(ref == -1) < len(S)


def test_minima_hopping_database(G, ctx, field):
    """Three hops of 256 replicas: the database grows, its structures are
    pairwise distinct by the oracle's RMSD, and sampled entries are minima
    of the oracle's force field with the energies the device reported."""
    from paper_2508_15522_gb300 import sampling as S
    sub, box, h, c32, grid = field
    mol = synth.chain_molecule()
    x0 = synth.flexible_positions(mol, sub, 256, seed=158)
    mh = S.MinimaHopping(ctx, grid, mol, x0, sub.tile, md_steps=300, dt=0.5, f_conv=1e-3, relax_steps=4000, seed=5)
    curve = [mh.hop() for _ in range(3)]
    counts = [c[1] for c in curve]
    assert counts[0] > 0 and counts == sorted(counts)
    assert (mh.db_x[..., 2] >= grid.floor).all()         # no accepted minimum below the grid
    db = mh.db_x[:40].astype(np.float64)
    assert (osamp.dup_of_xyz(db, sub.tile, 0.1) == -1).all()
    fn = odyn.make_force_fn(c32, ("C", "P", "L"), box.origin, h, mol)
    E, F, _ = fn(db[:8])
    assert np.allclose(E, mh.db_E[:8], atol=1e-4 * mol.n)
    assert (np.sqrt((F * F).sum((1, 2))) < 1e-3 + 5e-4).all()
    mh.close()
