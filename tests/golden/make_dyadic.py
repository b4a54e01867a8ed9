"""Writes dyadic_mixtures.json: noise-free linear mixtures that are exact in fp32.

Each case is a library S whose entries are k/64 (k integer in 13..38, i.e.
reflectances 0.2-0.6) and abundances that are dyadic fractions summing to 1.
Every product and sum in y = S^T x is then exact in binary32, so the observed
spectrum carries no rounding.  By the linear mixing model (Sec. 2.1, eq.
LinearMixing) with E = 0 and a library of full column rank, x is the unique
minimiser of the criterion (eq. UnconstrainedProblem) and satisfies the
constraints of Sec. 2.2 (eqs. NonNegativity, SumToOne), so the expected FCLS
answer is x itself.  No solver is involved in writing this file.
"""
import json
import os

import numpy as np


def main():
    rng = np.random.Generator(np.random.PCG64(1402_2518))
    cases = []
    for L, x in [(16, [0.5, 0.25, 0.125, 0.125]),
                 (24, [0.375, 0.25, 0.1875, 0.125, 0.0625]),
                 (32, [0.5, 0.5, 0.0, 0.0, 0.0, 0.0]),
                 (12, [1.0, 0.0, 0.0]),
                 (40, [0.25] * 4 + [0.0] * 4)]:
        P = len(x)
        while True:
            K = rng.integers(13, 39, size=(P, L))
            if np.linalg.matrix_rank(K.astype(float)) == P:
                break
        cases.append(dict(L=L, P=P, S_num=K.tolist(), S_den=64,
                          sigma=1.0 / 128, x=x))
    out = dict(
        source="Sec. 2.1 eq. LinearMixing with E = 0; Sec. 2.2 eqs. "
               "NonNegativity and SumToOne: an exact mixture by a full-rank "
               "library is its own FCLS minimiser",
        cases=cases)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "dyadic_mixtures.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
