"""Host logic of the sampling loop (paper_2508_15522_gb300/sampling.py), no
GPU: which relaxations count as minima, and how minima hopping treats
replicas that left the grid (library calls faked where a device is needed)."""
import numpy as np


def test_sampling_accepts_only_converged_in_grid_finite_relaxations():
    import __graft_entry__ as g
    g.build()
    from paper_2508_15522_gb300 import gridff as G
    from paper_2508_15522_gb300 import sampling as S
    st = np.array([0, G.REP_CONVERGED, G.REP_CONVERGED | G.REP_BELOW, G.REP_CONVERGED | G.REP_NONFINITE,
                   G.REP_BELOW, G.REP_CONVERGED | G.REP_STEPLIMIT, G.REP_STEPLIMIT, G.REP_CONVERGED | G.REP_ABORTED],
                  np.int32)
    assert S.accepted(st).tolist() == [False, True, False, False, False, True, False, True]
    # with the final structures: judged by the floor, not by the status bit
    x = np.zeros((8, 2, 3))
    x[:, :, 2] = 1.0
    x[5, 1, 2] = -0.01                                    # one atom of replica 5 ends below
    assert S.accepted(st, x, 0.0).tolist() == [False, True, True, False, False, False, False, True]
    b = S.Batch(np.zeros((3, 7)), np.array([-1.0, -0.995, -0.98]), np.array([True, True, True]), 0.0, 0.0)
    assert S.hits(b, -1.0).tolist() == [True, True, False]


def test_minima_hopping_restarts_replicas_that_left_the_grid(monkeypatch):
    """Host logic of the hopping loop with the library calls faked: a
    replica whose relaxed structure ends below the grid floor contributes no
    minimum and starts the next hop from its initial structure; one that
    only passed below on the way (status bit) and ended above is a minimum;
    the others keep their relaxed state."""
    import types
    import __graft_entry__ as g
    g.build()
    from paper_2508_15522_gb300 import gridff as G
    from paper_2508_15522_gb300 import sampling as S
    n_rep, n_at, z0 = 5, 2, 0.0

    class FakeReps:
        def __init__(self, ctx, mols, tof):
            self.x = np.zeros(3 * n_rep * n_at, np.float32)
            self.v = np.zeros_like(self.x)

        def set_state(self, x, v=None):
            self.x = np.array(x, np.float32)
            self.v = np.zeros_like(self.x) if v is None else np.array(v, np.float32)

        def get_state(self):
            return self.x.copy(), self.v.copy()

        def positions(self):
            return self.x.reshape(-1, 3).copy()

        def fire_state(self):
            c, b = G.REP_CONVERGED, G.REP_BELOW
            st = np.array([c, c | b, b, c, c | b], np.int32)
            return {"status": st, "energy": np.array([-1.0, -5.0, 0.0, -2.0, -3.0])}

        def close(self):
            pass

    def relax(ctx, grid, reps, n, fire, check=False):
        x = reps.x.reshape(n_rep, n_at, 3)
        x[:, :, 0] += 1.0                    # every replica moves
        x[[1, 2], 0, 2] = z0 - 0.5           # replicas 1 and 2 end with an atom below the floor
        reps.x = x.ravel()
        reps.v = np.full_like(reps.v, 0.5)

    fake = types.SimpleNamespace(Replicas=FakeReps, fire_params=lambda **kw: None, langevin=lambda *a, **k: None,
                                 relax=relax, rmsd_unique_xyz=lambda ctx, X, tile, thr: -np.ones(len(X), np.int32),
                                 REP_CONVERGED=G.REP_CONVERGED, REP_BELOW=G.REP_BELOW,
                                 REP_NONFINITE=G.REP_NONFINITE)
    monkeypatch.setattr(S, "G", fake)
    x0 = np.ones((n_rep, n_at, 3), np.float32) * np.arange(1, n_rep + 1, dtype=np.float32)[:, None, None]
    grid = types.SimpleNamespace(origin=(0.0, 0.0, z0 - 0.8), floor=z0)
    mh = S.MinimaHopping(None, grid, types.SimpleNamespace(n=n_at), x0, (1.0, 1.0))
    t, unique, acc = mh.hop()
    assert (unique, acc) == (3, 3) and mh.below == [2]
    assert mh.db_E.tolist() == [-3.0, -2.0, -1.0]           # -5.0 eV ended below the floor: no minimum
    x, v = mh.reps.get_state()
    x, v = x.reshape(x0.shape), v.reshape(x0.shape)
    assert np.array_equal(x[[1, 2]], x0[[1, 2]]) and (v[[1, 2]] == 0).all()
    kept = [0, 3, 4]
    assert np.array_equal(x[kept][..., 0], x0[kept][..., 0] + 1.0) and np.array_equal(x[kept][..., 1:], x0[kept][..., 1:])
    assert (v[kept] == 0.5).all()
