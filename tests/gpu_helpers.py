"""Shared helpers of the GPU parity tests (oracle references and tolerances)."""
import numpy as np

from oracle import assemble, iga1d


def oracle_matrix(d, p, n, alpha, beta):
    return assemble.galerkin_kron(d, p, n, alpha, beta)


def abs_matvec_bound(A, w):
    """(|A| |w|)_i: the scale of the rounding error of any summation order of A w."""
    return abs(A) @ np.abs(w)


def kron_rows(d, p, n, alpha, beta, w, rows):
    """Selected entries of A w for the printed Kronecker form, evaluated row by row from the
    oracle's 1D matrices (for sizes whose sparse matrix does not fit in memory)."""
    M, A, S = iga1d.matrices(p, n)
    At = A.T
    m = n + p - 2
    nper = m ** d
    W = w.reshape(d, *([m] * d))
    out = np.zeros(len(rows))
    absout = np.zeros(len(rows))
    if d == 2:
        curl = [[(M, S), (-At, A)], [(-A, At), (S, M)]]
        div = [[(S, M), (A, At)], [(At, A), (M, S)]]
    else:
        curl = [[[(M, M, S), (M, S, M)], [(-At, A, M)], [(-At, M, A)]],
                [[(-A, At, M)], [(S, M, M), (M, M, S)], [(-M, At, A)]],
                [[(-A, M, At)], [(-M, A, At)], [(S, M, M), (M, S, M)]]]
        div = [[[(S, M, M)], [(A, At, M)], [(A, M, At)]],
               [[(At, A, M)], [(M, S, M)], [(M, A, At)]],
               [[(At, M, A)], [(M, At, A)], [(M, M, S)]]]
        # negative first factor encodes the printed minus sign
    for k, r in enumerate(rows):
        c = r // nper
        idx = np.unravel_index(r % nper, [m] * d)
        tot, atot = 0.0, 0.0
        for c2 in range(d):
            if d == 2:
                terms = [(alpha, curl[c][c2]), (beta, div[c][c2])]
            else:
                terms = [(alpha, t) for t in curl[c][c2]] + [(beta, t) for t in div[c][c2]]
            for coef, mats in terms:
                # each 1D row is banded: contract over its nonzero window only
                rowv = [mats[l][idx[l], :] for l in range(d)]
                nz = [np.nonzero(v)[0] for v in rowv]
                sub = W[c2][np.ix_(*nz)]
                rv = [rowv[l][nz[l]] for l in range(d)]
                if d == 2:
                    t = np.einsum("i,j,ij->", rv[0], rv[1], sub)
                    at = np.einsum("i,j,ij->", np.abs(rv[0]), np.abs(rv[1]), np.abs(sub))
                else:
                    t = np.einsum("i,j,k,ijk->", rv[0], rv[1], rv[2], sub)
                    at = np.einsum("i,j,k,ijk->", *[np.abs(x) for x in rv], np.abs(sub))
                tot += coef * t
                atot += abs(coef) * at
        out[k] = tot
        absout[k] = atot
    return out, absout
