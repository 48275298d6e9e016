"""Second-quantised Hamiltonian on small determinant spaces (test helper).

Independent of the oracle: H is applied to a determinant written as an
ordered string of creation operators (spin-up before spin-down, increasing
index inside a spin; Sec. "Internal representation of determinants"), with
every fermionic sign counted by moving operators one position at a time:

    H = sum_{pq,s} h_pq a+_{ps} a_{qs}
        + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}

Spin orbitals are numbered so = s * norb + p, which is the ordering above.
"""
from __future__ import annotations

import numpy as np


def eri_full(eri_packed, norb):
    """Unpack 8-fold packed chemists' integrals into a dense 4-index array."""
    def tri(a, b):
        hi, lo = np.maximum(a, b), np.minimum(a, b)
        return hi * (hi + 1) // 2 + lo

    i = np.arange(norb, dtype=np.int64)
    pq = tri(i[:, None], i[None, :])
    idx = tri(pq[:, :, None, None], pq[None, None, :, :])
    return np.asarray(eri_packed)[idx]


def annihilate(state, i):
    """a_i on an ordered tuple; returns (sign, new tuple) or None."""
    if i not in state:
        return None
    k = state.index(i)
    return (-1) ** k, state[:k] + state[k + 1:]


def create(state, i):
    """a+_i on an ordered tuple: put i in front, then move it to its place."""
    if i in state:
        return None
    k = sum(1 for x in state if x < i)
    return (-1) ** k, state[:k] + (i,) + state[k:]


def apply_h(state, h, g, norb):
    """H|state> as a dict {ordered tuple: amplitude}."""
    out = {}
    nso = 2 * norb

    def add(st, v):
        out[st] = out.get(st, 0.0) + v

    for q in list(state):
        r1 = annihilate(state, q)
        s1, st1 = r1
        sq, pq_ = divmod(q, norb)
        for p in range(sq * norb, (sq + 1) * norb):
            r2 = create(st1, p)
            if r2 is None:
                continue
            s2, st2 = r2
            add(st2, s1 * s2 * h[p - sq * norb, pq_])
    # two-body: a+_p a+_r a_s a_q, with p,q of one spin and r,s of one spin
    for q in list(state):
        r1 = annihilate(state, q)
        s1, st1 = r1
        sig, qo = divmod(q, norb)
        for s in list(st1):
            r2 = annihilate(st1, s)
            s2, st2 = r2
            tau, so_ = divmod(s, norb)
            for r in range(tau * norb, (tau + 1) * norb):
                r3 = create(st2, r)
                if r3 is None:
                    continue
                s3, st3 = r3
                ro = r - tau * norb
                for p in range(sig * norb, (sig + 1) * norb):
                    r4 = create(st3, p)
                    if r4 is None:
                        continue
                    s4, st4 = r4
                    po = p - sig * norb
                    add(st4, 0.5 * s1 * s2 * s3 * s4 * g[po, qo, ro, so_])
    return out


def det_to_state(det, norb):
    """uint64[2, nint] determinant -> ordered tuple of spin orbitals."""
    st = []
    for s in range(2):
        for p in range(norb):
            if (int(det[s, p // 64]) >> (p % 64)) & 1:
                st.append(s * norb + p)
    return tuple(st)


def dense_h(dets, h, eri_packed, norb):
    """<I|H|J> for every pair of ``dets`` (uint64[n, 2, nint])."""
    g = eri_full(eri_packed, norb)
    states = [det_to_state(d, norb) for d in dets]
    index = {st: i for i, st in enumerate(states)}
    n = len(states)
    Hm = np.zeros((n, n))
    for j, st in enumerate(states):
        for st2, v in apply_h(st, h, g, norb).items():
            i = index.get(st2)
            if i is not None:
                Hm[i, j] += v
    return Hm
