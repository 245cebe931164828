"""Pin of the sparse-numerator restatement (oracle/sparse_numerator.py) to
the definition of the Cox coordinate derivatives (oracle.cox_terms, itself
pinned to brute-force risk sets).  CPU only."""
import numpy as np
import pytest
import scipy.sparse

import oracle
from paper_2204_08183_gb300 import synth


@pytest.mark.parametrize("seed,n_times,binary,density", [(1, 15, True, 0.3), (2, 400, False, 0.2),
                                                         (3, 5, False, 0.6), (4, 1000, True, 0.05)])
def test_sparse_numerator_equals_definition(seed, n_times, binary, density):
    d = synth.cohort_small(400, 6, seed, n_times=n_times, censor_frac=0.35, density=density)
    X = d["X"]
    if binary:
        X = (X != 0).astype(np.float64)
    beta = d["beta"] * 0.7
    Xs = scipy.sparse.csc_matrix(X)
    for j in range(6):
        ref = oracle.cox_terms(d["time"], d["status"], X, beta, j)
        got = oracle.cox_terms_sparse_numerator(d["time"], d["status"], Xs, beta, j)
        np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-11)


def test_empty_column_and_last_group():
    d = synth.cohort_small(60, 3, 5, n_times=8, censor_frac=0.3)
    X = np.zeros((60, 3))
    X[-3:, 1] = [1.0, 2.0, -1.0]          # nonzeros only in the last rows (last group)
    X[::7, 2] = 1.0
    beta = np.array([0.0, 0.2, -0.3])
    for j in range(3):
        ref = oracle.cox_terms(d["time"], d["status"], X, beta, j)
        got = oracle.cox_terms_sparse_numerator(d["time"], d["status"], X, beta, j)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
    # an all-zero column has l' = l'' = 0
    _, g1, g2 = oracle.cox_terms_sparse_numerator(d["time"], d["status"], X, beta, 0)
    assert g1 == 0.0 and g2 == 0.0
