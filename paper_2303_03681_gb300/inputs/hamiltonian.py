"""Synthetic Hamiltonians as Pauli sums.

Molecular part: the second-quantised electronic Hamiltonian of the paper's
"Unitary coupled cluster" subsection (one-body ``h`` and two-body ``g``
integrals), written in chemists' notation with spin summed explicitly,

    H = sum_{pq,s} h_pq a+_{ps} a_{qs}
        + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs},

with random integrals standing in for the PySCF ones the paper uses
(h_pq ~ N(0,1) symmetric, (pq|rs) ~ N(0, 0.1^2) with the 8-fold symmetry of
real orbitals).  Spin orbitals are interleaved (qubit 2p = p-up,
2p+1 = p-down) and mapped to qubits by Jordan-Wigner,
a_j = (Z_0 ... Z_{j-1}) (X_j + i Y_j) / 2 with |1> = occupied.

The mapping works on Pauli strings held in the symplectic form
X^x Z^z (bit vectors x, z packed in 64-bit words): the product of two such
strings is (-1)^{|z1 & x2|} X^{x1^x2} Z^{z1^z2}, and X Z = -i Y converts the
result to ordinary I/X/Y/Z strings at the end.
"""

from dataclasses import dataclass

import numpy as np

OP_I, OP_X, OP_Y, OP_Z = 0, 1, 2, 3
OP_CHARS = "IXYZ"

_BYTE_POPCOUNT = np.array([bin(i).count("1") for i in range(256)], dtype=np.uint8)


@dataclass
class PauliSum:
    """sum_k coeffs[k] * P_k with P_k = ops[k, 0] (x) ... (x) ops[k, n-1].

    ``ops`` is (n_terms, n_qubits) uint8 with 0=I, 1=X, 2=Y, 3=Z; an all-I row
    is a constant.  Coefficients are real (the operator is Hermitian).
    """

    n_qubits: int
    ops: np.ndarray
    coeffs: np.ndarray

    @property
    def n_terms(self) -> int:
        return int(self.ops.shape[0])

    def strings(self):
        return ["".join(OP_CHARS[o] for o in row) for row in self.ops]


# ----------------------------------------------------------------------------
# symplectic Pauli strings
# ----------------------------------------------------------------------------

def _n_words(n: int) -> int:
    return (n + 63) // 64


def _bit_tables(n: int):
    """Per-site word tables: e[j] = bit j, lt[j] = bits < j, le[j] = bits <= j."""
    w = _n_words(n)
    e = np.zeros((n, w), dtype=np.uint64)
    lt = np.zeros((n, w), dtype=np.uint64)
    for j in range(n):
        e[j, j // 64] = np.uint64(1) << np.uint64(j % 64)
    acc = np.zeros(w, dtype=np.uint64)
    for j in range(n):
        lt[j] = acc
        acc = acc | e[j]
    le = lt | e
    return e, lt, le


def _popcount(words: np.ndarray) -> np.ndarray:
    """Popcount summed over the last axis of a uint64 array."""
    b = np.ascontiguousarray(words).view(np.uint8)
    return _BYTE_POPCOUNT[b].reshape(words.shape[:-1] + (-1,)).sum(axis=-1, dtype=np.int64)


def _ladder_factor(idx, dagger, tables):
    """The two symplectic terms of a JW ladder operator for each index in idx.

    a_j  = 1/2 X^{e_j} Z^{lt_j} - 1/2 X^{e_j} Z^{le_j}
    a+_j = 1/2 X^{e_j} Z^{lt_j} + 1/2 X^{e_j} Z^{le_j}
    Returns (x, [z_0, z_1], [c_0, c_1]).
    """
    e, lt, le = tables
    x = e[idx]
    return x, (lt[idx], le[idx]), (0.5, 0.5 if dagger else -0.5)


def _expand_products(factors, weight):
    """Expand prod_k (sum_b c_kb X^{x_k} Z^{z_kb}) for vectors of index tuples.

    factors: list of (x, (z0, z1), (c0, c1)) with x, z of shape (K, W).
    weight:  (K,) complex prefactor.
    Returns (x, z, coef) with x, z of shape (K * 2^len, W).
    """
    nf = len(factors)
    xs, zs, cs = [], [], []
    for combo in range(1 << nf):
        bits = [(combo >> (nf - 1 - k)) & 1 for k in range(nf)]
        x_acc = factors[0][0].copy()
        z_acc = factors[0][1][bits[0]].copy()
        coef = weight * factors[0][2][bits[0]]
        sign = np.zeros(weight.shape[0], dtype=np.int64)
        for k in range(1, nf):
            xk = factors[k][0]
            zk = factors[k][1][bits[k]]
            sign += _popcount(z_acc & xk)
            x_acc ^= xk
            z_acc ^= zk
            coef = coef * factors[k][2][bits[k]]
        coef = np.where(sign & 1, -coef, coef)
        xs.append(x_acc)
        zs.append(z_acc)
        cs.append(coef)
    return np.concatenate(xs), np.concatenate(zs), np.concatenate(cs)


def _to_standard(x, z, coef):
    """X^x Z^z -> ordinary Pauli string: X Z = -i Y on every site with x=z=1."""
    ny = _popcount(x & z)
    phase = np.array([1.0, -1.0j, -1.0, 1.0j])[ny % 4]
    return coef * phase


class _Accumulator:
    """Sums coefficients of equal symplectic strings across chunks."""

    def __init__(self, n: int):
        self.n = n
        self.w = _n_words(n)
        self.keys = []
        self.vals = []

    def add(self, x, z, coef):
        if x.shape[0] == 0:
            return
        key, val = self._reduce(np.concatenate([x, z], axis=1), coef)
        self.keys.append(key)
        self.vals.append(val)

    def _reduce(self, rows, coef):
        rows = np.ascontiguousarray(rows, dtype=np.uint64)
        void = rows.view(np.dtype((np.void, rows.dtype.itemsize * rows.shape[1]))).ravel()
        uniq, inv = np.unique(void, return_inverse=True)
        re = np.bincount(inv, weights=coef.real, minlength=uniq.shape[0])
        im = np.bincount(inv, weights=coef.imag, minlength=uniq.shape[0])
        out = uniq.view(np.uint64).reshape(-1, rows.shape[1])
        return out, re + 1j * im

    def result(self):
        if not self.keys:
            return np.zeros((0, 2 * self.w), np.uint64), np.zeros(0, complex)
        return self._reduce(np.concatenate(self.keys), np.concatenate(self.vals))


def _symplectic_to_ops(rows, n):
    w = _n_words(n)
    x, z = rows[:, :w], rows[:, w:]
    ops = np.zeros((rows.shape[0], n), dtype=np.uint8)
    for j in range(n):
        word, bit = j // 64, np.uint64(j % 64)
        xb = ((x[:, word] >> bit) & np.uint64(1)).astype(np.uint8)
        zb = ((z[:, word] >> bit) & np.uint64(1)).astype(np.uint8)
        # (x,z): (1,0)=X, (1,1)=Y, (0,1)=Z
        ops[:, j] = np.where(xb & zb, OP_Y, np.where(xb, OP_X, np.where(zb, OP_Z, OP_I)))
    return ops


def ops_to_symplectic(ops: np.ndarray):
    """I/X/Y/Z strings (T, n) uint8 -> packed (x, z) bit words, each (T, W)
    uint64 with site j at bit j % 64 of word j // 64 (X: x, Y: x and z, Z: z)."""
    ops = np.asarray(ops, dtype=np.uint8)
    T, n = ops.shape
    w = _n_words(n)
    out = []
    for bits in ((ops == OP_X) | (ops == OP_Y), (ops == OP_Y) | (ops == OP_Z)):
        pad = np.zeros((T, 64 * w), dtype=bool)
        pad[:, :n] = bits
        packed = np.packbits(pad, axis=1, bitorder="little")  # (T, 8 w) bytes, bit j of byte j // 8
        out.append(np.ascontiguousarray(packed).view("<u8").astype(np.uint64).reshape(T, w))
    return out[0], out[1]


def symplectic_to_ops(x: np.ndarray, z: np.ndarray, n: int) -> np.ndarray:
    """Inverse of ``ops_to_symplectic``."""
    return _symplectic_to_ops(np.concatenate([x, z], axis=1), n)


def fermion_terms_to_paulis(n_so, terms, tol=1e-12):
    """JW-map a list of fermionic monomials to an exact complex Pauli sum.

    ``terms`` is an iterable of (weights (K,), [(idx (K,), dagger), ...]):
    K monomials weight * prod_k op_k, operators left to right.
    Returns (ops (T, n) uint8, complex coefficients (T,)), zeros dropped.
    """
    tables = _bit_tables(n_so)
    acc = _Accumulator(n_so)
    for weight, ops in terms:
        weight = np.asarray(weight, dtype=complex)
        if weight.shape[0] == 0:
            continue
        factors = [_ladder_factor(np.asarray(idx), dag, tables) for idx, dag in ops]
        x, z, coef = _expand_products(factors, weight)
        acc.add(x, z, _to_standard(x, z, coef))
    rows, vals = acc.result()
    keep = np.abs(vals) > tol
    rows, vals = rows[keep], vals[keep]
    ops = _symplectic_to_ops(rows, n_so)
    order = np.lexsort(ops.T[::-1])
    return ops[order], vals[order]


# ----------------------------------------------------------------------------
# molecular Hamiltonian
# ----------------------------------------------------------------------------

def random_integrals(n_orb: int, rng: np.random.Generator, g_scale: float = 0.1):
    """h_pq ~ N(0,1) symmetric and (pq|rs) ~ N(0, g_scale^2) with 8-fold symmetry.

    Every symmetry class of (pq|rs) takes one independent draw, so each
    entry keeps variance g_scale^2.
    """
    h = rng.normal(0.0, 1.0, (n_orb, n_orb))
    h = np.triu(h) + np.triu(h, 1).T
    raw = rng.normal(0.0, g_scale, (n_orb,) * 4)
    p, q, r, s = np.indices((n_orb,) * 4)
    pq_hi, pq_lo = np.maximum(p, q), np.minimum(p, q)
    rs_hi, rs_lo = np.maximum(r, s), np.minimum(r, s)
    pq = pq_hi * n_orb + pq_lo
    rs = rs_hi * n_orb + rs_lo
    swap = pq < rs
    a_hi = np.where(swap, rs_hi, pq_hi)
    a_lo = np.where(swap, rs_lo, pq_lo)
    b_hi = np.where(swap, pq_hi, rs_hi)
    b_lo = np.where(swap, pq_lo, rs_lo)
    g = raw[a_hi, a_lo, b_hi, b_lo]
    return h, g


def jw_molecular_hamiltonian(h: np.ndarray, g: np.ndarray, constant: float = 0.0,
                             chunk: int = 1 << 19) -> PauliSum:
    """Jordan-Wigner Pauli sum of the spin-summed molecular Hamiltonian."""
    n_orb = h.shape[0]
    n_so = 2 * n_orb
    terms = []
    # one-body: h_pq a+_{p s} a_{q s}
    p, q = np.meshgrid(np.arange(n_orb), np.arange(n_orb), indexing="ij")
    p, q = p.ravel(), q.ravel()
    for s in (0, 1):
        w = h[p, q]
        nz = w != 0.0
        terms.append((w[nz], [(2 * p[nz] + s, True), (2 * q[nz] + s, False)]))
    # two-body: 1/2 (pq|rs) a+_{p s} a+_{r t} a_{s' t} a_{q s}, chunked over p
    idx = np.arange(n_orb)
    _, qq, rr, ss = np.meshgrid([0], idx, idx, idx, indexing="ij")
    qq, rr, ss = qq.ravel(), rr.ravel(), ss.ravel()
    for pv in range(n_orb):
        w_all = 0.5 * g[pv, qq, rr, ss]
        for s1 in (0, 1):
            for s2 in (0, 1):
                P = 2 * pv + s1
                Q = 2 * qq + s1
                R = 2 * rr + s2
                S = 2 * ss + s2
                keep = (R != P) & (S != Q) & (w_all != 0.0)
                if not np.any(keep):
                    continue
                Pk = np.full(int(keep.sum()), P)
                terms.append((w_all[keep], [(Pk, True), (R[keep], True), (S[keep], False), (Q[keep], False)]))
    ops, vals = fermion_terms_to_paulis(n_so, _chunked(terms, chunk))
    if np.max(np.abs(vals.imag), initial=0.0) > 1e-9:
        raise ValueError("Hamiltonian is not Hermitian: imaginary Pauli coefficient")
    coeffs = vals.real.copy()
    if constant != 0.0:
        ident = ~ops.any(axis=1)
        if ident.any():
            coeffs[np.argmax(ident)] += constant
        else:
            ops = np.vstack([np.zeros((1, n_so), np.uint8), ops])
            coeffs = np.concatenate([[constant], coeffs])
    return PauliSum(n_so, ops, coeffs)


def fermion_monomial_map(n_so: int, ops, tol: float = 1e-14):
    """JW-map K fermionic monomials separately, sharing one set of strings.

    ``ops`` lists the operators left to right as (idx (K,), dagger); monomial
    k is prod_m op_m[k].  Returns (strings, row_ptr, cols, weights): the
    distinct Pauli strings (T, n_so) uint8 and a CSR map with
    monomial k = sum_{e in row_ptr[k]:row_ptr[k+1]} weights[e] * strings[cols[e]]
    (complex weights, entries of one row in increasing column order).
    """
    tables = _bit_tables(n_so)
    idx0 = np.asarray(ops[0][0])
    K = int(idx0.shape[0])
    if K == 0:
        return (np.zeros((0, n_so), np.uint8), np.zeros(1, np.int64), np.zeros(0, np.int32),
                np.zeros(0, complex))
    factors = [_ladder_factor(np.asarray(idx), dag, tables) for idx, dag in ops]
    x, z, coef = _expand_products(factors, np.ones(K, dtype=complex))
    coef = _to_standard(x, z, coef)
    mono = np.tile(np.arange(K, dtype=np.int64), 1 << len(ops))  # _expand_products stacks combination-major
    rows = np.ascontiguousarray(np.concatenate([x, z], axis=1), dtype=np.uint64)
    void = rows.view(np.dtype((np.void, rows.dtype.itemsize * rows.shape[1]))).ravel()
    uniq, first, inv = np.unique(void, return_index=True, return_inverse=True)
    T = int(uniq.shape[0])
    key = mono * T + inv.reshape(-1)
    ukey, kinv = np.unique(key, return_inverse=True)
    w = (np.bincount(kinv, weights=coef.real, minlength=ukey.shape[0])
         + 1j * np.bincount(kinv, weights=coef.imag, minlength=ukey.shape[0]))
    keep = np.abs(w) > tol
    ukey, w = ukey[keep], w[keep]
    row_of, col_of = ukey // T, ukey % T
    used, cols = np.unique(col_of, return_inverse=True)
    strings = _symplectic_to_ops(rows[first[used]], n_so)
    row_ptr = np.searchsorted(row_of, np.arange(K + 1)).astype(np.int64)
    return strings, row_ptr, cols.astype(np.int32), w


def _chunked(terms, chunk):
    for weight, ops in terms:
        k = weight.shape[0]
        for lo in range(0, k, chunk):
            hi = min(k, lo + chunk)
            yield weight[lo:hi], [(np.asarray(i)[lo:hi], d) for i, d in ops]


def hf_bits(n_so: int, n_electrons: int) -> np.ndarray:
    """Hartree-Fock reference: the lowest ``n_electrons`` spin orbitals occupied."""
    bits = np.zeros(n_so, dtype=np.uint8)
    bits[:n_electrons] = 1
    return bits


# ----------------------------------------------------------------------------
# 1D local Pauli sums
# ----------------------------------------------------------------------------

def random_local_pauli_sum(n: int, n_terms: int, rng: np.random.Generator,
                           next_nearest: bool = True) -> PauliSum:
    """``n_terms`` distinct strings drawn uniformly from the pool of non-identity
    single-site, nearest-neighbour (j, j+1) and, if ``next_nearest``,
    next-nearest-neighbour (j, j+2) Pauli products; coefficients ~ N(0, 1)."""
    pool = []
    for j in range(n):
        for a in (1, 2, 3):
            pool.append(((j, a),))
    for d in ((1, 2) if next_nearest else (1,)):
        for j in range(n - d):
            for a in (1, 2, 3):
                for b in (1, 2, 3):
                    pool.append(((j, a), (j + d, b)))
    if n_terms > len(pool):
        raise ValueError(f"only {len(pool)} distinct local strings on {n} sites")
    pick = np.sort(rng.choice(len(pool), size=n_terms, replace=False))
    ops = np.zeros((n_terms, n), dtype=np.uint8)
    for row, k in enumerate(pick):
        for site, op in pool[k]:
            ops[row, site] = op
    coeffs = rng.normal(0.0, 1.0, n_terms)
    return PauliSum(n, ops, coeffs)
