"""Auto-fit of the reference library (Sec. 2.4, "Estimation of
degeneracies"), plain numpy / scipy in fp64 (test infrastructure, like the
rest of ``oracle``; the CUDA library shares no code with it).

For each spectrum S_n of the library, the other spectra S' = S without S_n
fit it in the least-squares sense, S_n = A'.S' + E:

* unconstrained (eq. UnconstrainedProblem): the residue E is the part of
  S_n orthogonal to the span of S' (unique even when S' is rank
  deficient; numpy's SVD least squares);
* non-negative (eq. UnconstrainedProblem under eq. NonNegativityConstraint):
  scipy's NNLS (Lawson-Hanson); the fit A'.S' is unique, the coefficients
  are unique when S' has full rank.

The spectra are not weighted (the database has no noise model).
"""
from __future__ import annotations

import numpy as np
import scipy.optimize


def autofit(S) -> dict:
    """S: (P, L) library.  Returns dict(resid_ls, resid_nn (P, L), coef_nn
    (P, P), row n = coefficients of the other spectra with 0 at n, rms_ls,
    rms_nn (P,)), all fp64."""
    S = np.asarray(S, dtype=np.float32).astype(np.float64)
    P, L = S.shape
    out = dict(resid_ls=np.empty((P, L)), resid_nn=np.empty((P, L)),
               coef_nn=np.zeros((P, P)), rms_ls=np.empty(P), rms_nn=np.empty(P))
    for n in range(P):
        others = [j for j in range(P) if j != n]
        A = S[others].T                       # L x (P - 1)
        y = S[n]
        a_ls = np.linalg.lstsq(A, y, rcond=None)[0]
        e_ls = y - A @ a_ls
        a_nn = scipy.optimize.nnls(A, y, maxiter=50 * P)[0]
        e_nn = y - A @ a_nn
        out["resid_ls"][n] = e_ls
        out["resid_nn"][n] = e_nn
        out["coef_nn"][n, others] = a_nn
        out["rms_ls"][n] = np.sqrt(np.mean(e_ls ** 2))
        out["rms_nn"][n] = np.sqrt(np.mean(e_nn ** 2))
    return out
