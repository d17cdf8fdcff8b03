"""The signed-feature cases of the GPU parity tests reach both branches of
Eq. 4's maximum (checked on the CPU with the oracle's cosine and codes)."""
import numpy as np
import pytest

from oracle import gift_oracle as O
from tests.signed_case import negative_terms, signed_case


@pytest.mark.parametrize("ma,db_ma", [(1, 1), (2, 1), (1, 2)])
def test_signed_case_has_both_kinds_of_negative_maxima(ma, db_ma):
    X, cb, Q, qoff, dbc, qc = signed_case(ma=ma, db_ma=db_ma)
    covered, partial = negative_terms(X, Q, dbc, qc)
    assert covered >= 5 and partial >= 50, (covered, partial)
    # Eq. 4 differs from the zero-floored maximum on this case: the literal
    # oracle has negative terms that a floor at 0 would remove
    S = O.fif_scores(Q, qoff, qc, X, dbc)
    assert (S < 0).any() or covered > 0


def test_signed_one_codeword_case_is_exact_match():
    X, cb, Q, qoff, dbc, qc = signed_case(K=1, N=60)
    assert (dbc == 0).all() and (qc == 0).all()
    assert np.allclose(O.fif_scores(Q, qoff, qc, X, dbc), O.exact_scores(Q, qoff, X), rtol=0, atol=1e-15)
    assert (O.exact_scores(Q, qoff, X) < 0).any()
