"""GPU parity of the batched relaxation layouts (unique-term flexible kernel
with warps-per-block, stencil-staging and work-queue variants), the
autotuner and CUDA-graph replay, against the oracle's FIRE."""
import numpy as np
import pytest

from oracle import dynamics as odyn
from oracle import grid as ogrid
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
    coefs = synth.random_coefficients(n, 3, seed=71, scale=(0.02, 0.01, 0.03))
    grid = G.grid_from_coefs(ctx, coefs, box.origin, h, 7)
    return sub, box, h, coefs.astype(np.float32).astype(np.float64), grid


@pytest.fixture(scope="module")
def uneven():
    """Templates of 10, 47 and 70 atoms with torsions, and an uneven replica
    list (the 128-atom maximum is covered by its own one-step case)."""
    mols = [synth.chain_molecule(), synth.random_flexible_molecule(47, 8, 3),
            synth.random_flexible_molecule(70, 10, 5)]
    tof = np.array([0, 2, 1, 1, 0, 2, 0, 1, 0], np.int32)
    return mols, tof


def _start(sub, mols, tof, seed):
    xs = []
    for r, t in enumerate(tof):
        xs.append(synth.flexible_positions(mols[t], sub, 1, seed=seed + r)[0])
    return [x.astype(np.float32) for x in xs]


CHECKPOINTS = (1, 5, 20)


def _oracle(field, mols, tof, x0, checkpoints=CHECKPOINTS):
    """Oracle FIRE positions of every replica after each checkpoint's number
    of steps (one trajectory per template, continued between checkpoints)."""
    sub, box, h, c32, grid = field
    out = {k: [None] * len(tof) for k in checkpoints}
    for t, mol in enumerate(mols):
        rows = [r for r in range(len(tof)) if tof[r] == t]
        if not rows:
            continue
        fn = odyn.make_force_fn(c32, ("C", "P", "L"), box.origin, h, mol)
        x = np.stack([x0[r] for r in rows]).astype(np.float64)
        v = np.zeros_like(x)
        state, done = None, 0
        for k in checkpoints:
            ref = odyn.fire_flexible(x, v, mol.mass, fn, k - done, odyn.FireParams(f_conv=0.0), state=state)
            x, v, done = ref["x"], ref["v"], k
            state = {key: ref[key] for key in ("dt", "alpha", "nplus", "status", "steps")}
            for j, r in enumerate(rows):
                out[k][r] = x[j]
    return out


@pytest.fixture(scope="module")
def refs(field, uneven):
    mols, tof = uneven
    x0 = _start(field[0], mols, tof, 81)
    return x0, _oracle(field, mols, tof, x0)


LAYOUTS = [dict(kernel=3, warps_per_block=w, cache_slots=S, queue=q, cache_global=0)
           for w, S, q in ((2, 0, 1), (4, 32, 1), (8, 64, 0), (4, 70, 0), (8, 16, 1))]
LAYOUTS += [dict(kernel=3, warps_per_block=w, cache_slots=0, queue=q, cache_global=1) for w, q in ((8, 1), (2, 0))]
LAYOUTS += [dict(kernel=2, warps_per_block=4, cache_slots=S, queue=0, cache_global=0) for S in (0, 48)]
TOL = {1: 2e-6, 5: 2e-5, 20: 2e-4}


def _relax_and_compare(G, ctx, grid, mols, tof, x0, ref, configure):
    for nsteps in CHECKPOINTS:
        reps = G.Replicas(ctx, mols, tof)
        configure(reps)
        reps.set_state(np.concatenate([x.ravel() for x in x0]))
        st, res = G.relax(ctx, grid, reps, nsteps, G.fire_params(f_conv=0.0))
        assert res.atom_evals == sum(mols[t].n for t in tof) * nsteps
        x, _ = reps.get_state()
        off = reps.atom_offset
        for r in range(len(tof)):
            xr = x[3 * off[r]:3 * off[r + 1]].reshape(-1, 3)
            assert np.abs(xr - ref[nsteps][r]).max() <= TOL[nsteps], (nsteps, r)
        assert (reps.fire_state()["steps"] == nsteps).all()
        reps.close()


@pytest.mark.parametrize("layout", LAYOUTS,
                         ids=lambda d: "k{kernel}-w{warps_per_block}-S{cache_slots}-q{queue}-g{cache_global}".format(**d))
def test_flex_terms_layouts_match_oracle(G, ctx, field, uneven, refs, layout):
    mols, tof = uneven
    x0, ref = refs
    _relax_and_compare(G, ctx, field[4], mols, tof, x0, ref,
                       lambda reps: reps.set_launch_config(G.LaunchConfig(lanes_per_replica=32, l2_window=0,
                                                                          **layout)))


def test_global_stencil_cache_rejected_where_it_does_not_apply(G, ctx, uneven):
    """cache_global belongs to the unique-term kernel without shared-memory
    slots: with slots, with another kernel, or with a value other than 0/1
    set_launch_config returns EINVAL."""
    mols, tof = uneven
    reps = G.Replicas(ctx, mols, tof)
    for bad in (dict(kernel=3, warps_per_block=4, cache_slots=16, queue=1, cache_global=1),
                dict(kernel=2, warps_per_block=4, cache_slots=0, queue=0, cache_global=1),
                dict(kernel=3, warps_per_block=4, cache_slots=0, queue=1, cache_global=2)):
        with pytest.raises(G.GridffError) as e:
            reps.set_launch_config(G.LaunchConfig(lanes_per_replica=32, l2_window=0, **bad))
        assert e.value.status == G.EINVAL
    reps.close()


def test_global_stencil_cache_changes_nothing_but_the_layout(G, ctx, field, uneven, refs):
    """The global stencil cache stores the same channel-combined values the
    gathers produce and the contraction reads them in the same order, so a
    relaxation and a Langevin run with and without it agree bit for bit."""
    mols, tof = uneven
    x0 = np.concatenate([x.ravel() for x in refs[0]])
    out = {}
    for gc in (0, 1):
        reps = G.Replicas(ctx, mols, tof)
        reps.set_launch_config(kernel=G.KERNEL_FLEX_TERMS, warps_per_block=4, cache_slots=0, queue=1,
                               cache_global=gc)
        reps.set_state(x0)
        G.relax(ctx, field[4], reps, 50, G.fire_params(f_conv=0.0))
        xr = reps.get_state()[0].copy()
        G.langevin(ctx, field[4], reps, 30, 1.0, 300.0, 0.01, 5)
        out[gc] = (xr, reps.get_state()[0].copy(), reps.fire_state()["energy"].copy())
        reps.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_flex_terms_largest_molecule_one_step(G, ctx, field):
    mol = synth.random_flexible_molecule(128, 12, 4)
    x0 = [synth.flexible_positions(mol, field[0], 1, seed=131)[0].astype(np.float32)]
    ref = _oracle(field, [mol], np.array([0]), x0, checkpoints=(1,))
    reps = G.Replicas(ctx, [mol], [0])
    reps.set_launch_config(kernel=G.KERNEL_FLEX_TERMS, warps_per_block=4, cache_slots=128, queue=1)
    reps.set_state(x0[0].ravel())
    G.relax(ctx, field[4], reps, 1, G.fire_params(f_conv=0.0))
    x, _ = reps.get_state()
    assert np.abs(x.reshape(-1, 3) - ref[1][0]).max() <= TOL[1]
    reps.close()


def test_flex_terms_energy_matches_eval(G, ctx, field, uneven):
    """The energy a relaxation reports equals gridff_eval at the final state."""
    sub, box, h, c32, grid = field
    mols, tof = uneven
    reps = G.Replicas(ctx, mols, tof)
    reps.set_launch_config(kernel=G.KERNEL_FLEX_TERMS, warps_per_block=4, cache_slots=32, queue=1)
    reps.set_state(np.concatenate([x.ravel() for x in _start(sub, mols, tof, 91)]))
    G.relax(ctx, grid, reps, 1, G.fire_params(f_conv=0.0))      # energy of the evaluated (start) state
    e_relax = reps.fire_state()["energy"]
    reps.set_state(np.concatenate([x.ravel() for x in _start(sub, mols, tof, 91)]))
    E, F, _ = G.eval(ctx, grid, reps)[:3]
    assert np.allclose(e_relax, E, atol=1e-5 * 128, rtol=1e-5)


def test_tuner_restores_state_and_picks_a_valid_layout(G, ctx, field, uneven, refs):
    sub, box, h, c32, grid = field
    mols, tof = uneven
    reps = G.Replicas(ctx, mols, tof)
    x0 = np.concatenate([x.ravel() for x in refs[0]])
    reps.set_state(x0)
    before = reps.get_state()
    best, log = G.tune(ctx, grid, reps, G.fire_params(f_conv=0.0), trial_steps=5)
    after = reps.get_state()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    assert len(log) >= 4 and max(t["atom_evals_per_s"] for t in log) > 0
    cfg = reps.launch_config()
    assert cfg.kernel == best.kernel and cfg.cache_slots == best.cache_slots
    reps.close()
    # relaxing with the tuned layout gives the oracle's trajectory
    _relax_and_compare(G, ctx, grid, mols, tof, refs[0], refs[1],
                       lambda r: r.set_launch_config(best))


def test_rigid_tuner_and_graph_replay_bitwise(G, ctx, field):
    """Rigid kernels are deterministic: a graph replay equals a direct call
    bit for bit, for the tuned layout."""
    sub, box, h, c32, grid = field
    mol = synth.c24h8o6_core()
    n_rep = 300
    com, quat = synth.rigid_poses(mol, sub, n_rep, seed=111)
    pose = np.concatenate([com, quat], 1).astype(np.float32).ravel()
    reps = G.Replicas(ctx, [mol], [0] * n_rep, rigid=True)
    reps.set_state(pose)
    best, log = G.tune(ctx, grid, reps, G.fire_params(f_conv=0.0), trial_steps=10)
    assert best.kernel in (G.KERNEL_RIGID_SUBWARP, G.KERNEL_RIGID_QUAD)
    G.relax(ctx, grid, reps, 50, G.fire_params(f_conv=0.0))
    x_direct, _ = reps.get_state()
    graph = G.RelaxGraph(ctx, grid, reps, 50, G.fire_params(f_conv=0.0))
    for _ in range(2):
        reps.set_state(pose)
        st, res = graph.launch()
        assert res.atom_evals == n_rep * mol.n * 50
        x_graph, _ = reps.get_state()
        assert np.array_equal(x_graph, x_direct)
    graph.close()
    reps.close()


def _rigid_state(reps):
    x, v = reps.get_state()
    fs = reps.fire_state()
    return x, v, fs


@pytest.mark.parametrize("blocks", [3, 7])
def test_rigid_time_sliced_schedule_bitwise(G, ctx, field, blocks):
    """With fewer resident warps than warp tasks, the sub-warp relaxation
    either splits tasks between two warps (head and tail, handed over
    through global memory; queue mode 2) or hands whole tasks out from an
    atomic queue (mode 1; mode 0 picks the queue when f_conv > 0).  The
    per-replica arithmetic is the same in every schedule, so the final
    state equals the uncapped run bit for bit, also for a continued call;
    convergence is counted once; a CUDA-graph replay of the split launch
    matches as well."""
    sub, box, h, c32, grid = field
    mol = synth.c24h8o6_core()
    n_rep, nsteps = 301, 150          # odd: the last warp task has one replica
    com, quat = synth.rigid_poses(mol, sub, n_rep, seed=141)
    pose = np.concatenate([com, quat], 1).astype(np.float32).ravel()
    base = dict(kernel=G.KERNEL_RIGID_SUBWARP, lanes_per_replica=16, warps_per_block=4, cache_slots=mol.n,
                l2_window=0)
    for f_conv in (0.0, 0.05):
        out = {}
        for cap, mode in ((0, 0), (blocks, 0), (blocks, 1), (blocks, 2)):
            reps = G.Replicas(ctx, [mol], [0] * n_rep, rigid=True)
            reps.set_launch_config(G.LaunchConfig(blocks=cap, queue=mode, **base))
            reps.set_state(pose)
            fp = G.fire_params(f_conv=f_conv)
            st, res = G.relax(ctx, grid, reps, nsteps, fp, check=False)
            first = (_rigid_state(reps), res.atom_evals, res.n_converged, res.max_steps)
            st, res = G.relax(ctx, grid, reps, 100, fp, flags=G.CONTINUE, check=False)
            out[cap, mode] = (first, (_rigid_state(reps), res.atom_evals, res.n_converged, res.max_steps))
            if cap and mode == 2 and f_conv == 0.0:
                graph = G.RelaxGraph(ctx, grid, reps, nsteps, fp)
                reps.set_state(pose)
                graph.launch()
                xg, _ = reps.get_state()
                assert np.array_equal(xg, out[cap, mode][0][0][0])
                graph.close()
            reps.close()
        ref = out[0, 0]
        for key, got in out.items():
            for (sa, ea, ca, ma), (sb, eb, cb, mb) in zip(ref, got):
                (xa, va, fa), (xb, vb, fb) = sa, sb
                assert np.array_equal(xa, xb) and np.array_equal(va, vb), key
                for k in ("dt", "alpha", "nplus", "status", "steps", "energy"):
                    assert np.array_equal(fa[k], fb[k]), (key, k)
                assert (ea, ca, ma) == (eb, cb, mb), key
        if f_conv == 0.0:
            assert ref[0][1] == n_rep * mol.n * nsteps and ref[0][2] == 0
        else:
            # the threshold lets part of the batch converge inside the window
            assert 0 < ref[0][2] < n_rep


def test_rigid_split_schedule_stops_on_abort_and_budget(G, ctx, field):
    """On the split schedule a tail never runs on after its head was
    stopped: with the abort flag set nothing moves; with a clock budget
    every replica ends with STEPLIMIT and the context stays usable."""
    sub, box, h, c32, grid = field
    mol = synth.c24h8o6_core()
    n_rep = 301
    com, quat = synth.rigid_poses(mol, sub, n_rep, seed=161)
    pose = np.concatenate([com, quat], 1).astype(np.float32).ravel()
    reps = G.Replicas(ctx, [mol], [0] * n_rep, rigid=True)
    reps.set_launch_config(G.LaunchConfig(kernel=G.KERNEL_RIGID_SUBWARP, lanes_per_replica=16, warps_per_block=4,
                                          cache_slots=mol.n, queue=2, blocks=3))
    reps.set_state(pose)
    ctx.set_abort(True)
    try:
        st, res = G.relax(ctx, grid, reps, 200, G.fire_params(f_conv=0.0), check=False)
    finally:
        ctx.set_abort(False)
    assert st == G.EABORTED
    fs = reps.fire_state()
    assert ((fs["status"] & G.REP_ABORTED) != 0).all() and (fs["steps"] == 0).all()
    x, _ = reps.get_state()
    assert np.array_equal(x, pose)
    st, res = G.relax(ctx, grid, reps, 10_000_000, G.fire_params(f_conv=0.0, clock_budget_s=0.05), check=False)
    assert st == G.ESTEPLIMIT
    fs = reps.fire_state()
    assert ((fs["status"] & G.REP_STEPLIMIT) != 0).all()
    assert (fs["steps"] < 10_000_000).all() and (fs["steps"] > 0).any()
    st, res = G.relax(ctx, grid, reps, 3, G.fire_params(f_conv=0.0))
    assert st == G.OK and res.atom_evals == n_rep * mol.n * 3
    reps.close()


def test_rigid_split_schedule_wait_is_bounded(G, ctx, field):
    """Test hook GRIDFF_TEST_NO_HANDOFF: the first parts of split tasks
    publish nothing, so every second part gives up after its bounded wait;
    the call returns ETIMEOUT, the replicas of split tasks keep the state of
    their first part, whole tasks finish, and the context stays usable."""
    sub, box, h, c32, grid = field
    mol = synth.c24h8o6_core()
    n_rep, nsteps = 301, 150
    com, quat = synth.rigid_poses(mol, sub, n_rep, seed=171)
    pose = np.concatenate([com, quat], 1).astype(np.float32).ravel()
    reps = G.Replicas(ctx, [mol], [0] * n_rep, rigid=True)
    reps.set_launch_config(G.LaunchConfig(kernel=G.KERNEL_RIGID_SUBWARP, lanes_per_replica=16, warps_per_block=4,
                                          cache_slots=mol.n, queue=2, blocks=3))
    reps.set_state(pose)
    st, res = G.relax(ctx, grid, reps, nsteps, G.fire_params(f_conv=0.0), flags=G.TEST_NO_HANDOFF, check=False)
    assert st == G.ETIMEOUT
    steps = reps.fire_state()["steps"]
    assert (steps <= nsteps).all() and (steps < nsteps).any() and (steps == nsteps).any()
    st, res = G.relax(ctx, grid, reps, 5, G.fire_params(f_conv=0.0))
    assert st == G.OK and res.atom_evals == n_rep * mol.n * 5
    reps.close()


def test_rigid_nve_time_sliced_schedule_bitwise(G, ctx, field):
    """Rigid NVE on the split schedule (block cap 3): positions, velocities,
    energies and the recorded energy trace equal the unsplit run bit for
    bit (the head hands its quaternion momentum on exactly)."""
    sub, box, h, c32, grid = field
    mol = synth.c24h8o6_core()
    n_rep, nsteps = 301, 150
    com, quat = synth.rigid_poses(mol, sub, n_rep, seed=151)
    pose = np.concatenate([com, quat], 1).astype(np.float32).ravel()
    g = np.random.default_rng(152)
    vel = (g.standard_normal((n_rep, 6)) * np.array([2e-3] * 3 + [5e-3] * 3)).astype(np.float32).ravel()
    out = []
    for cap in (0, 3):
        reps = G.Replicas(ctx, [mol], [0] * n_rep, rigid=True)
        if cap:
            reps.set_launch_config(G.LaunchConfig(kernel=G.KERNEL_RIGID_SUBWARP, lanes_per_replica=16,
                                                  warps_per_block=4, cache_slots=mol.n, blocks=cap))
        reps.set_state(pose, vel)
        st, trace = G.run(ctx, grid, reps, nsteps, dt=1.0, record_every=10)
        x, v = reps.get_state()
        fs = reps.fire_state()
        out.append((x, v, fs["status"], fs["energy"], trace))
        reps.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    assert np.isfinite(out[0][4]).all()


def test_flex_graph_replay_matches_direct(G, ctx, field, uneven):
    sub, box, h, c32, grid = field
    mols, tof = uneven
    x0 = np.concatenate([x.ravel() for x in _start(sub, mols, tof, 121)])
    reps = G.Replicas(ctx, mols, tof)
    reps.set_launch_config(kernel=G.KERNEL_FLEX_TERMS, warps_per_block=4, cache_slots=32, queue=1)
    reps.set_state(x0)
    G.relax(ctx, grid, reps, 30, G.fire_params(f_conv=0.0))
    x_direct, _ = reps.get_state()
    graph = G.RelaxGraph(ctx, grid, reps, 30, G.fire_params(f_conv=0.0))
    reps.set_state(x0)
    graph.launch()
    x_graph, _ = reps.get_state()
    # shared-memory atomics sum in a run-dependent order: FP32 rounding only
    assert np.abs(x_graph - x_direct).max() < 1e-4
    graph.close()
    reps.close()


def test_bad_launch_configs_are_rejected(G, ctx, uneven):
    mols, tof = uneven
    reps = G.Replicas(ctx, mols, tof)
    with pytest.raises(G.GridffError):
        reps.set_launch_config(kernel=G.KERNEL_RIGID_SUBWARP)        # flexible replicas
    with pytest.raises(G.GridffError):
        reps.set_launch_config(kernel=G.KERNEL_FLEX_TERMS, warps_per_block=3)
    with pytest.raises(G.GridffError):
        reps.set_launch_config(kernel=G.KERNEL_FLEX_TERMS, warps_per_block=4, cache_slots=500)
    reps.close()


def test_edge_sizes_flexible_one_and_two_atoms(G, ctx, field):
    """Molecules of one and two atoms (no nonbonded pair, one excluded pair)
    in the unique-term kernel, against the oracle."""
    sub, box, h, c32, grid = field
    g = synth.rng(171)
    mols = []
    for n in (1, 2):
        els = ["C", "O"][:n]
        R = np.array([synth.ELEMENTS[e][0] for e in els]); eps = np.array([synth.ELEMENTS[e][1] for e in els])
        xyz = np.array([[0.0, 0.0, 0.0], [1.2, 0.0, 0.0]])[:n]
        bonds = np.array([[0, 1]], np.int32) if n == 2 else np.zeros((0, 2), np.int32)
        m = synth.Molecule(els, xyz, np.zeros(n), R, eps, np.array([12.0, 16.0])[:n], bonds=bonds,
                           bond_k=np.array([20.0])[:len(bonds)], bond_r0=np.array([1.25])[:len(bonds)])
        mols.append(m)
    tof = np.array([0, 1, 0, 1], np.int32)
    x0 = [(mols[t].xyz + [g.uniform(0, 5), g.uniform(0, 5), box.origin[2] + 3.0]).astype(np.float32) for t in tof]
    reps = G.Replicas(ctx, mols, tof)
    reps.set_launch_config(kernel=G.KERNEL_FLEX_TERMS, warps_per_block=8, cache_slots=0, queue=1)
    reps.set_state(np.concatenate([x.ravel() for x in x0]))
    G.relax(ctx, grid, reps, 5, G.fire_params(f_conv=0.0))
    x, _ = reps.get_state()
    off = reps.atom_offset
    for r, t in enumerate(tof):
        fn = odyn.make_force_fn(c32, ("C", "P", "L"), box.origin, h, mols[t])
        ref = odyn.fire_flexible(x0[r][None].astype(np.float64), np.zeros((1,) + x0[r].shape), mols[t].mass, fn, 5,
                                 odyn.FireParams(f_conv=0.0))
        assert np.abs(x[3 * off[r]:3 * off[r + 1]].reshape(-1, 3) - ref["x"][0]).max() < 2e-5
    reps.close()


def test_rigid_largest_molecule_subwarp(G, ctx, field):
    """A 128-atom rigid body (the template maximum) takes the 32-lane,
    4-atoms-per-lane instance of the sub-warp kernel."""
    sub, box, h, c32, grid = field
    mol = synth.rigid_molecule(128, 181)
    com, quat = synth.rigid_poses(mol, sub, 5, seed=182)
    pose = np.concatenate([com, quat], 1).astype(np.float32)
    reps = G.Replicas(ctx, [mol], [0] * 5, rigid=True)
    cfg = reps.launch_config()
    assert cfg.kernel == G.KERNEL_RIGID_SUBWARP and cfg.lanes_per_replica == 32
    reps.set_state(pose.ravel())
    G.relax(ctx, grid, reps, 3, G.fire_params(f_conv=0.0))
    x, _ = reps.get_state()
    body = mol.xyz.astype(np.float32).astype(np.float64)
    fn = odyn.make_force_fn(c32, ("C", "P", "L"), box.origin, h, mol, intra=False)
    ref = odyn.fire_rigid(pose[:, :3].astype(np.float64), pose[:, 3:].astype(np.float64), np.zeros((5, 3)),
                          np.zeros((5, 3)), body, mol.mass, fn, 3, odyn.FireParams(f_conv=0.0))
    xg = odyn.rigid_positions(x.reshape(5, 7)[:, :3].astype(np.float64), x.reshape(5, 7)[:, 3:].astype(np.float64),
                              body)
    assert np.abs(xg - odyn.rigid_positions(ref["com"], ref["quat"], body)).max() < 5e-5
    reps.close()
