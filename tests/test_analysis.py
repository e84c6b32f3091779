"""Post-decoding statistics, pinned by brute-force ML decoding on tiny codes."""
import itertools

import numpy as np

from paper_1204_0556_gb300 import analysis as A
from paper_1204_0556_gb300 import inputs as I


def _codewords(code):
    """All codewords of a small code by enumeration of the null space of H over GF(2)."""
    H = code.dense().astype(np.int64)
    words = []
    for bits in itertools.product([0, 1], repeat=code.n):
        c = np.array(bits)
        if not (H @ c % 2).any():
            words.append(c)
    return np.array(words)


def test_ml_lower_bound_counts_only_true_ml_errors(oracle_mod):
    code = I.gallager_code(12, 3, 6, 0)
    C = _codewords(code)
    llr = I.awgn_llr(code, 0.0, 400, 17).astype(np.float64)
    r = oracle_mod.decode(code.row_ptr, code.col_idx, code.n, llr, mu=3.0, rho=1.9, eps=1e-8, max_iter=5000)
    flagged = A.ml_lower_bound_errors(code, llr, r["bits"])
    ml_choice = np.argmin(llr @ C.T, axis=1)  # ML decision: the codeword minimizing gamma^T c
    ml_error = C[ml_choice].any(axis=1)
    assert flagged.sum() >= 5
    assert np.all(ml_error[flagged])           # every flagged frame is an ML error
    assert flagged.sum() <= ml_error.sum()     # hence a lower bound on ML errors
    decoder_error = r["bits"].any(axis=1)
    assert flagged.sum() <= decoder_error.sum()


def test_ml_lower_bound_hand_cases():
    code = I.code_from_rows(4, [[0, 1, 2], [1, 2, 3]])  # codewords include 0110 and 1011
    llr = np.array([[1.0, -2.0, -2.0, 1.0],   # 0110 decoded, gamma^T c = -4 < 0 -> ML error
                    [1.0, 2.0, 2.0, 1.0],     # 0110 decoded, gamma^T c = 4 > 0 -> not counted
                    [1.0, -2.0, -2.0, 1.0]])  # 0100 decoded: not a codeword -> not counted
    bits = np.array([[0, 1, 1, 0], [0, 1, 1, 0], [0, 1, 0, 0]])
    assert A.ml_lower_bound_errors(code, llr, bits).tolist() == [True, False, False]
    assert A.syndromes(code, bits).tolist() == [[0, 0], [0, 0], [1, 1]]


def test_error_rates_and_pseudocodewords():
    bits = np.array([[0, 0, 0, 0], [0, 1, 0, 0], [1, 1, 0, 0]])
    iters = np.array([5, 100, 300])
    e = A.error_rates(bits, iters)
    assert e["wer"] == 2 / 3 and e["ber"] == 3 / 12
    assert e["iters_correct"] == 5 and e["iters_erroneous"] == 200
    x = np.array([[0.0, 1.0, 0.5, 0.5], [0.0, 0.0, 0.0, 1.0]])
    s = A.pseudocodeword_summary(x)
    assert s["frames_fractional"] == 1 and s["fractional_coords_mean"] == 2
    assert sum(s["value_histogram"]) == 2


def test_gallager_ensemble():
    ens = I.gallager_ensemble(1002, 3, 6, 3)
    assert len(ens) == 3
    for c in ens:
        assert (c.n, c.m, c.E) == (1002, 501, 3006)
        assert set(c.check_degrees.tolist()) == {6} and set(c.var_degrees.tolist()) == {3}
    assert not np.array_equal(ens[0].col_idx, ens[1].col_idx)
