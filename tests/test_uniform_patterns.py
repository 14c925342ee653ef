"""The node kernel's compiled sparsity patterns (generated at build time by csrc/gen_uniform.cpp from the
library's coupling tables) against the oracle's matrices, which come from sphere quadrature
(oracle/sh.py) and share nothing with the library: for l_max = 1..5 every nonzero of
Omega^x, Omega^y, Omega^z (and the diagonal) lies in R's pattern, every nonzero of A^a in beta_a's and
every nonzero of |A^a| = W |Lambda| W^T (numpy eigh) in |beta_a|'s.  A pattern that missed an entry
would drop a coupling; the set-up refuses the node kernel for matrices outside the patterns, so the
superset property is what makes the kernel apply the operator of Sec. 2.2.  Also: no pattern is much
larger than the oracle's (no dense fill)."""
import os
import re

import numpy as np
import pytest

from oracle import sh


@pytest.fixture(scope="module")
def patterns():
    from paper_2501_05110_gb300 import build
    os.makedirs(build.OUT, exist_ok=True)
    build._generate_patterns()  # the current generator (a host program; no GPU needed)
    text = open(build.PATTERNS).read()
    out = {}
    for m in re.finditer(r"template <> struct UniK<(\d+)> \{(.*?)\n\};", text, re.S):
        L = int(m.group(1))
        body = m.group(2)
        pats = {}
        for name, arr in re.findall(r"static constexpr unsigned char (pat\w+)\[\d+\]\[2\] = \{(.*?)\};", body):
            pats[name] = {tuple(map(int, p)) for p in re.findall(r"\{(\d+),(\d+)\}", arr)}
        out[L] = pats
    return out


def _nz(M, rel=1e-12):
    M = np.asarray(M)
    cut = rel * np.abs(M).max()
    return {(int(i), int(j)) for i, j in zip(*np.nonzero(np.abs(M) > cut))}


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5])
def test_patterns_contain_oracle_matrices(patterns, L):
    T = sh.tables(L)
    n = (L + 1) ** 2
    P = patterns[L]
    diag = {(i, i) for i in range(n)}
    want_R = _nz(T["Om"][0]) | _nz(T["Om"][1]) | _nz(T["Om"][2]) | diag
    assert want_R <= P["patR"]
    for a in range(3):
        A = np.asarray(T["A"][a])
        assert _nz(A) | diag <= P[f"patB{a}"], a
        w, V = np.linalg.eigh(A)
        absA = V @ np.diag(np.abs(w)) @ V.T
        assert _nz(absA) <= P[f"patA{a}"], a
        # no dense fill: at most the oracle's count plus the diagonal
        assert len(P[f"patA{a}"]) <= len(_nz(absA) | diag), a
        assert len(P[f"patB{a}"]) == len(_nz(A) | diag), a
    assert len(P["patR"]) == len(want_R)
