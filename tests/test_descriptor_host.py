"""gridff_molecule_descriptor is a host computation: checked on the CPU,
entry by entry, against a numpy restatement of its definition in the header
(inertia eigenvalues by numpy's symmetric eigensolver instead of the
library's trigonometric closed form)."""
import numpy as np
import pytest

from paper_2508_15522_gb300 import synth


def _reference(mol):
    x = np.asarray(mol.xyz, np.float64)
    m = np.asarray(mol.mass, np.float64)
    q = np.asarray(mol.q, np.float64)
    n, M = len(m), m.sum()
    r = x - (m[:, None] * x).sum(0) / M
    r2 = (r * r).sum(1)
    I = (m[:, None, None] * (r2[:, None, None] * np.eye(3) - r[:, :, None] * r[:, None, :])).sum(0)
    ev = np.sort(np.clip(np.linalg.eigvalsh(I), 0.0, None))
    cls = np.digitize(m, [4, 13, 15, 17])
    d = np.zeros(64)
    d[0] = n / 128
    d[1:6] = np.bincount(cls, minlength=5) / n
    d[6] = q.sum()
    d[7] = np.linalg.norm((q[:, None] * r).sum(0)) / 10
    d[8:11] = np.sqrt(ev / M) / 5
    d[11] = np.sqrt((m * r2).sum() / M) / 5
    d[12] = np.sqrt(r2.max()) / 10
    d[13] = len(mol.torsions) / 12
    return d


def _molecules():
    lin = synth.Molecule(["C", "O", "H"], np.array([[0.0, 0, 0], [1.2, 0, 0], [-1.0, 0, 0]]),
                         np.array([0.3, -0.4, 0.1]), np.array([1.9, 1.7, 1.4]), np.array([0.07, 0.05, 0.04]),
                         np.array([12.011, 15.999, 1.008]))
    one = synth.Molecule(["O"], np.array([[0.5, -0.2, 3.0]]), np.array([0.0]), np.array([1.7]),
                         np.array([0.05]), np.array([15.999]))
    return [synth.c24h8o6_core(), synth.chain_molecule(), synth.random_flexible_molecule(60, 10, 5),
            synth.random_flexible_molecule(120, 12, 7), lin, one]


@pytest.mark.parametrize("k", range(6))
def test_descriptor_matches_its_definition(k):
    import __graft_entry__ as g
    g.build()
    from paper_2508_15522_gb300 import gridff
    mol = _molecules()[k]
    got = gridff.molecule_descriptor(mol).astype(np.float64)
    want = _reference(mol)
    assert np.abs(got - want).max() < 2e-6 * max(1.0, np.abs(want).max()), (got[:14], want[:14])
