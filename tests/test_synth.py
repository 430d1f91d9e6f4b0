"""Input generator: the close-atom check used for cells above 300 atoms (periodic k-d tree
plus the exact minimum image) finds exactly the atoms the all-pairs check finds."""
import numpy as np
import pytest

from paper_2606_19557_gb300 import synth


def _all_pairs(fr, cell, dmin):
    n = fr.shape[0]
    bad = np.zeros(n, bool)
    for i0 in range(0, n, 512):
        i1 = min(n, i0 + 512)
        df = fr[None, :, :] - fr[i0:i1, None, :]
        df -= np.round(df)
        d = df @ cell
        d2 = np.einsum("ijk,ijk->ij", d, d)
        idx = np.arange(i0, i1)
        d2[idx - i0, idx] = np.inf
        bad[i0:i1] |= (d2 < dmin * dmin).any(axis=1)
    return np.nonzero(bad)[0]


@pytest.mark.parametrize("kind,n,sigma", [("fcc", 5000, 0.45), ("bcc", 320, 0.5), ("fcc", 900, 0.4),
                                          ("bcc", 2000, 0.45)])
def test_tree_close_atoms_equals_all_pairs(kind, n, sigma):
    rng = np.random.default_rng(n)
    a = synth.FCC_A if kind == "fcc" else synth.BCC_A
    frac, cell = synth._lattice(kind, synth._supercell_reps(4 if kind == "fcc" else 2, n), a)
    e = rng.uniform(-0.03, 0.03, size=(3, 3))
    cell = cell @ (np.eye(3) + 0.5 * (e + e.T))
    pos = frac @ cell + rng.normal(scale=sigma, size=(frac.shape[0], 3))
    fr = pos @ np.linalg.inv(cell)
    got = synth._close_atoms_tree(fr, cell, 1.2)
    assert got.size > 10
    assert np.array_equal(got, _all_pairs(fr, cell, 1.2))
