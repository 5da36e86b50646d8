"""The oracle's whole-block J/K (used to sample large configurations) against
its full unique-quartet J/K build on small bases, for a symmetric and an
antisymmetric density.  The full build is pinned against quadrature,
closed forms and symmetries elsewhere; the block routine evaluates the
definitions J_mn = sum (mn|ls) D_ls, K_mn = sum (ml|sn) D_ls directly.
CPU only."""
import numpy as np

import synth


def test_blocks_equal_full_build(oracle_lib):
    orc = oracle_lib
    mol, bas = synth.small_cluster(4, 551, max_depth=3)
    ob = orc.OBasis(mol, bas)
    n = ob.nbf
    D = synth.density(n, 5, 1)
    A = synth.hermitian_component(n, 3, complex_=False)
    A = A - A.T                                     # antisymmetric
    J, K = orc.jk_real(ob, [D, A])
    nc = [(int(l) + 1) * (int(l) + 2) // 2 for l in ob.L]
    bfo = np.concatenate([[0], np.cumsum(nc)])
    pairs = [(0, 0), (ob.nsh - 1, 0), (5, 2), (7, 7), (ob.nsh - 1, ob.nsh - 2)]
    out = orc.jk_blocks(ob, [D, A], [p[0] for p in pairs], [p[1] for p in pairs])
    for (a, b), (Jb, Kb) in zip(pairs, out):
        for q in range(2):
            assert np.abs(Jb[q] - J[q][bfo[a]:bfo[a + 1], bfo[b]:bfo[b + 1]]).max() < 1e-12
            assert np.abs(Kb[q] - K[q][bfo[a]:bfo[a + 1], bfo[b]:bfo[b + 1]]).max() < 1e-12
