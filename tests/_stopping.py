"""Why an early-exit decode may stop at another iteration than the oracle.

The stopping test of Section 3.3 compares two residual sums with eps^2 E.  The
GPU forms them from FP32 state, the oracle in FP64, so on a frame whose
residual crosses the threshold at iteration k by less than the FP32 error of
the sum, the two stop one or more iterations apart.  Any other difference in
iteration count means the two stopping tests differ.
"""
import numpy as np


def assert_stop_near_threshold(oracle_mod, code, llr_row, k_gpu: int, k_ref: int, *, mu: float, rho: float,
                               eps: float, band: float = 2.0) -> float:
    """Run the oracle for k = min(k_gpu, k_ref) iterations on one frame and
    check that max(R_p, R_d) / (eps^2 E) there lies within a factor `band` of 1:
    one decoder stopped at k and the other did not, which only rounding near
    the threshold explains.  Returns the ratio."""
    k = int(min(k_gpu, k_ref))
    assert k >= 1, (k_gpu, k_ref)
    r = oracle_mod.decode(code.row_ptr, code.col_idx, code.n, np.asarray(llr_row, dtype=np.float64)[None, :],
                          mu=mu, rho=rho, eps=0.0, max_iter=k)
    E = int(code.row_ptr[-1])
    q = max(float(r["rp"][0]), float(r["rd"][0])) / (eps * eps * E)
    assert 1.0 / band <= q <= band, (k_gpu, k_ref, q)
    return q
