"""The quality report's permutation of a pattern, P A P^T, checked on CPU tensors against the
definition (entry (i, j) of the result is entry (perm[i], perm[j]) of A) and against the oracle's
bandwidth and profile of the same ordering."""
import numpy as np
import pytest

import oracle
from paper_1610_08128_gb300 import synth

torch = pytest.importorskip("torch")


def test_permute_csr_is_p_a_pt():
    from paper_1610_08128_gb300 import quality

    for g in [synth.grid((9, 7), seed=1), synth.random_graph(300, 700, 2, diagonal=True), synth.knn_mesh(400, 3, 3),
              synth.csr_from_edges(5, [], [])]:
        perm = oracle.rcm(g.n, g.rowptr, g.colidx)
        rp, ci = quality.permute_csr(torch.from_numpy(g.rowptr), torch.from_numpy(g.colidx), torch.from_numpy(perm))
        rp, ci = rp.numpy(), ci.numpy()
        assert rp[-1] == g.nnz and rp[0] == 0
        pos = np.empty(g.n, np.int64)
        pos[perm] = np.arange(g.n)
        for i in range(g.n):
            v = perm[i]
            want = sorted(pos[g.colidx[g.rowptr[v]:g.rowptr[v + 1]]].tolist())
            assert ci[rp[i]:rp[i + 1]].tolist() == want
        # bandwidth and profile of the permuted pattern in its own (identity) order equal the
        # oracle's for the ordering
        ident = np.arange(g.n, dtype=np.int32)
        assert oracle.bandwidth_profile(g.n, rp, ci, ident) == oracle.bandwidth_profile(g.n, g.rowptr, g.colidx, perm)
