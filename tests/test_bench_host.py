"""Host bookkeeping of bench.py's error report against the FP64 pairwise
reference (`grid_error_vs_pairwise`), with the library calls faked: the fake
returns the oracle's own values, shifted on one molecule, so the report's
per-molecule, per-atom and force maxima are known in closed form."""
import types

import numpy as np

import bench
from oracle import substrate as osub
from paper_2508_15522_gb300 import synth


def test_grid_error_report_bookkeeping():
    sub = synth.rocksalt_slab(a=5.64, ncell=2, layers=2, charge=0.7)
    m1, m2 = synth.chain_molecule(), synth.random_flexible_molecule(12, 2, 3)
    items = [(m1, m1.xyz + [0.0, 0.0, sub.z_top + 3.0]), (m2, m2.xyz + [1.0, 1.0, sub.z_top + 4.0]),
             (m1, m1.xyz + [2.0, 0.0, sub.z_top + 3.5])]
    x = np.concatenate([v for _, v in items]).astype(np.float32)
    mols = [m for m, _ in items]
    Er, Fr = osub.pairwise_reference(x.astype(np.float64), np.concatenate([m.q for m in mols]),
                                     np.concatenate([m.R for m in mols]), np.concatenate([m.eps for m in mols]), sub)
    lo, hi = m1.n, m1.n + m2.n                 # atoms of the second molecule
    dE, dF = 1e-3, 2e-3

    class FakeReps:
        def __init__(self, ctx, mols, tof):
            self.n = mols[0].n

        def template_factors(self, t):
            return np.zeros((self.n, 3), np.float32)

        def close(self):
            pass

    def eval_points(ctx, grid, pts, qpl):
        assert pts.shape == qpl.shape == (len(x), 3)
        assert np.array_equal(pts, x)
        E = Er.copy()
        F = Fr.copy()
        E[lo:hi] += dE
        F[lo, 1] -= dF
        S = np.zeros(len(x), np.int32)
        S[-1] = 2
        return E, F, S

    G = types.SimpleNamespace(Replicas=FakeReps, eval_points=eval_points)
    r = bench.grid_error_vs_pairwise(G, None, None, sub, items, "three molecules")
    assert r["molecules"] == 3 and r["atoms"] == len(x) and r["points_flagged"] == 1
    assert abs(r["max_abs_dE_per_molecule_eV"] - m2.n * dE) < 1e-12
    assert abs(r["max_abs_dE_per_atom_eV"] - dE) < 1e-15
    assert abs(r["max_abs_dF_eV_per_A"] - dF) < 1e-15


def test_amortised_gain_charges_training_and_credits_its_hits():
    """The learned arm's amortised rate: training-data relaxations and
    training time charged, their hits credited; break-even where the
    amortised rate equals the random-start rate."""
    import bench
    out = {"batches": 4, "random": {"hits_per_s": 100.0},
           "mlp": {"hits": 4000, "wall_s": 4.0}}
    a = bench.amortised_gain(out, train_hits=250, gen_s=2.5, train_s=1.0)
    assert a["proposal_batch_hits"] == 1000 and a["proposal_batch_s"] == 1.0
    assert abs(a["hits_per_s_after_4_batches"] - (250 + 4000) / (3.5 + 4.0)) < 1e-12
    assert abs(a["gain_after_4_batches"] - (4250 / 7.5) / 100.0) < 1e-12
    n = a["break_even_batches"]
    assert abs((250 + n * 1000) / (3.5 + n * 1.0) - 100.0) < 1e-9
    assert bench.amortised_gain(out, 400, 2.5, 1.0)["break_even_batches"] == 0.0   # ahead from the start
    out["mlp"]["hits"] = 400                      # proposals no better than random starts: no break-even
    assert bench.amortised_gain(out, 250, 2.5, 1.0)["break_even_batches"] is None


def test_clock_summary_keeps_the_timed_window():
    """Clock samples count only when they arrived inside the timed region;
    throttle reasons are read from the same samples."""
    import bench
    c = bench.ClockSampler(0)
    row = lambda mhz, slow: [0, str(mhz), "2070", "900", "x", "Active" if slow else "Not Active",
                             "Not Active", "Not Active", "Not Active"]
    c.rows = [(0.5, row(1200, True)), (1.1, row(2070, False)), (1.4, row(2060, False)), (3.0, row(900, True))]
    c.window = (1.0, 1.5)
    s = c.summary()
    assert s["samples"] == 2 and s["sm_mhz"] == 2065 and s["reasons"] == [] and s["sm_max_mhz"] == 2070
    c.window = (2.0, 2.5)          # nothing inside: the last samples around it
    assert c.summary()["samples"] == 3
    c.rows = []
    assert c.summary()["reasons"] == ["unsampled"]
