"""Dense hierarchy Liouvillian built from Kronecker superoperators (numpy), for pinning the oracle.

This is a third, independent statement of Eq. (HEOM) of arXiv 1803.03498: instead of the
element-wise Kronecker-delta loops of the oracle, every term is a matrix acting on the row-major
vectorisation vec(A) (vec(X A Y) = (X kron Y^T) vec(A)):

    commutator   -i (H kron 1 - 1 kron H^T)
    V^x          V kron 1 - 1 kron V^T
    V^o          V kron 1 + 1 kron V^T
    V^x V^x      (V^x)^2

Two gauges are available:
  form="paper"  : up  +i s+ V^x,  down  s- (i c V^x + delta_k0 lambda nu V^o)   (real c, rescaling)
  form="common" : up  -i V^x,     down  -i n (c~ V kron 1 - c~* 1 kron V^T)      (textbook form,
                  c~_0 = lambda nu (cot(beta nu / 2) - i), c~_k = c_k; no rescaling)
The two agree on sigma_0 because sigma_n -> (-1)^|n| sigma_n maps one onto the other; a wrong
relative sign or a dropped factor i in either makes them disagree.

Tuples are enumerated here with itertools (own order); ``index`` maps tuple -> block index.
"""
from __future__ import annotations

import itertools

import numpy as np


def enumerate_tuples(M: int, D: int):
    out = []
    for L in range(D + 1):
        for c in itertools.product(range(L + 1), repeat=M):
            if sum(c) == L:
                out.append(tuple(c))
    return out


def build(H_rad, mode_state, gamma, c, lamnu, delta_state, D, terminator=True, rescale=True, form="paper"):
    """H_rad: [N, N] complex, rad/fs.  Per mode: state, gamma, c (real), lamnu.  delta_state: [N]
    terminator coefficient summed per state.  Returns (L dense [nN^2, nN^2], tuples, index)."""
    N = H_rad.shape[0]
    eye = np.eye(N)
    mode_v = [eye[s] for s in mode_state]
    bath_terms = [(delta_state[s], eye[s]) for s in range(N) if delta_state[s] != 0.0]
    return build_general(H_rad, mode_v, gamma, c, lamnu, bath_terms, D, terminator, rescale, form)


def build_general(H_rad, mode_v, gamma, c, lamnu, bath_terms, D, terminator=True, rescale=True, form="paper"):
    """As build, for diagonal coupling operators: mode l couples through V_l = diag(mode_v[l]);
    bath_terms: [(Delta_b, diagonal of V_b)], the terminator adds -Delta_b (V_b^x)^2."""
    N = H_rad.shape[0]
    M = len(gamma)
    I = np.eye(N)
    tuples = enumerate_tuples(M, D)
    index = {t: k for k, t in enumerate(tuples)}
    nn = N * N
    L = np.zeros((len(tuples) * nn, len(tuples) * nn), dtype=complex)
    comm = np.kron(H_rad, I) - np.kron(I, H_rad.T)
    P = [np.diag(np.asarray(v, dtype=float)) for v in mode_v]
    Vx = [np.kron(P[l], I) - np.kron(I, P[l].T) for l in range(M)]
    Vo = [np.kron(P[l], I) + np.kron(I, P[l].T) for l in range(M)]
    term = np.zeros((nn, nn), dtype=complex)
    if terminator:
        for delta, v in bath_terms:
            Vb = np.diag(np.asarray(v, dtype=float))
            X = np.kron(Vb, I) - np.kron(I, Vb.T)
            term += delta * (X @ X)
    for t, u in index.items():
        blk = slice(u * nn, (u + 1) * nn)
        g = sum(t[l] * gamma[l] for l in range(M))
        L[blk, blk] += -1j * comm - g * np.eye(nn) - term
        for l in range(M):
            ac = abs(c[l])
            if sum(t) < D:
                tp = list(t); tp[l] += 1
                v = index[tuple(tp)]
                if form == "paper":
                    f = np.sqrt((t[l] + 1) * ac) if (rescale and ac > 1e-300) else 1.0
                    L[blk, v * nn:(v + 1) * nn] += 1j * f * Vx[l]
                else:
                    L[blk, v * nn:(v + 1) * nn] += -1j * Vx[l]
            if t[l] >= 1:
                tm = list(t); tm[l] -= 1
                v = index[tuple(tm)]
                if form == "paper":
                    f = np.sqrt(t[l] / ac) if (rescale and ac > 1e-300) else float(t[l])
                    L[blk, v * nn:(v + 1) * nn] += f * (1j * c[l] * Vx[l] + lamnu[l] * Vo[l])
                else:
                    ct = c[l] - 1j * lamnu[l]
                    L[blk, v * nn:(v + 1) * nn] += -1j * t[l] * (ct * np.kron(P[l], I) - np.conj(ct) * np.kron(I, P[l].T))
    return L, tuples, index


def build_from_oracle(model, form="paper", rescale=None, terminator=None):
    """Dense Liouvillian for an ``OracleModel`` using its exported coefficients."""
    from oracle.oracle import lib  # noqa: F401  (ensures the oracle library is built)
    md = model.modes()
    N = model.N
    H = np.asarray(model.H, dtype=complex) * 1.8836515673088532e-4
    delta_state = np.zeros(N)
    for b, bath in enumerate(model.baths):
        delta_state[bath.state] += md["delta"][b]
    return build(H, md["state"], md["gamma"], md["c"], md["lamnu"], delta_state, model.D,
                 terminator=model.terminator if terminator is None else terminator,
                 rescale=model.rescale if rescale is None else rescale, form=form)


def to_vec(re, im, oracle_tuples, index):
    """Oracle-ordered state [n, N, N] -> Liouvillian vector in this module's tuple order."""
    n, N, _ = re.shape
    v = np.zeros(n * N * N, dtype=complex)
    for u in range(n):
        k = index[tuple(int(x) for x in oracle_tuples[u])]
        v[k * N * N:(k + 1) * N * N] = (re[u] + 1j * im[u]).reshape(-1)
    return v


def from_vec(v, oracle_tuples, index, N):
    n = len(oracle_tuples)
    out = np.zeros((n, N, N), dtype=complex)
    for u in range(n):
        k = index[tuple(int(x) for x in oracle_tuples[u])]
        out[u] = v[k * N * N:(k + 1) * N * N].reshape(N, N)
    return out
