"""Post-decoding statistics (host-side, on the outputs of liblpdec).

* ``ml_lower_bound_errors``: the paper's estimate of a lower bound on the
  maximum-likelihood word error rate (Section 5.1, the [1057,813] code
  experiment): a decoding error counts as an ML error only when the rounded
  output satisfies every check and is more likely than the transmitted word.
  With the all-zeros word sent and gamma_i = log W(y_i|0)/W(y_i|1), a codeword
  c is more likely than 0 exactly when gamma^T c < 0.
* ``pseudocodeword_summary``: for frames whose LP solution is fractional, the
  number of fractional coordinates and the values they take (LP decoding fails
  on pseudocodewords, Sections 1 and 5.1).
* ``error_rates``: word and bit error rates against the all-zeros word, and the
  iteration counts split into correctly and wrongly decoded frames (the
  statistics of the random-ensemble experiment, Section 5.1).
"""
from __future__ import annotations

import numpy as np


def syndromes(code, bits: np.ndarray) -> np.ndarray:
    """Per-frame parity of every check of the hard decisions ([frames x m], 0/1)."""
    bits = np.atleast_2d(bits).astype(np.int64)
    out = np.zeros((bits.shape[0], code.m), dtype=np.int64)
    for j in range(code.m):
        cols = code.col_idx[code.row_ptr[j]:code.row_ptr[j + 1]]
        out[:, j] = bits[:, cols].sum(axis=1) & 1
    return out


def ml_lower_bound_errors(code, llr: np.ndarray, bits: np.ndarray) -> np.ndarray:
    """Boolean per frame: the decoder erred AND an ML decoder would err too.

    The all-zeros word was sent, so a frame is in error when any bit is 1.  If
    its rounded output b is a codeword with gamma^T b < 0, b is more likely
    than the transmitted word and ML decoding fails as well."""
    llr = np.atleast_2d(np.asarray(llr, dtype=np.float64))
    bits = np.atleast_2d(bits).astype(np.int64)
    err = bits.any(axis=1)
    is_codeword = ~syndromes(code, bits).any(axis=1)
    more_likely = (llr * bits).sum(axis=1) < 0.0
    return err & is_codeword & more_likely


def pseudocodeword_summary(x: np.ndarray, tol: float = 1e-2) -> dict:
    """Fractional coordinates of x (entries farther than tol from 0 and 1)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    frac = np.minimum(x, 1.0 - x) > tol
    per_frame = frac.sum(axis=1)
    vals = x[frac]
    return {
        "frames_fractional": int((per_frame > 0).sum()),
        "fractional_coords_mean": float(per_frame[per_frame > 0].mean()) if (per_frame > 0).any() else 0.0,
        "value_histogram": np.histogram(vals, bins=10, range=(0.0, 1.0))[0].tolist(),
    }


def error_rates(bits: np.ndarray, iters: np.ndarray) -> dict:
    """WER, BER and mean iterations (all, correct, erroneous) for the all-zeros word."""
    bits = np.atleast_2d(bits)
    iters = np.asarray(iters)
    err = bits.any(axis=1)
    ok = ~err
    return {
        "frames": int(len(err)),
        "wer": float(err.mean()),
        "ber": float(bits.mean()),
        "iters_mean": float(iters.mean()),
        "iters_correct": float(iters[ok].mean()) if ok.any() else None,
        "iters_erroneous": float(iters[err].mean()) if err.any() else None,
    }
