"""Reduced density matrices of a GPU state (Methods, "The DMET method").

The DMET fragment energy and electron count are functions of the 1-RDM
<a+_p a_q> and the 2-RDM <a+_p a+_q a_r a_s> of the fragment's VQE state.
Under the Jordan-Wigner map each element is a complex combination of at
most 16 Pauli strings, so one evaluation of the per-string expectation
values (the energy kernels, environments shared through one trie over the
union of the strings) gives all of them; the device then forms every
element as a weighted row sum (``mps_observables_eval``).

Kinds (interleaved spin orbitals, qubit 2p + s; n_so = 2 n_orb):

* ``"1rdm"``  gamma[P, Q] = <a+_P a_Q>                  (n_so, n_so)
* ``"2rdm"``  Gamma[P, Q, R, S] = <a+_P a+_Q a_R a_S>   (n_so,)*4
* ``"D"``     D[p, q] = sum_s <a+_{ps} a_{qs}>          (n_orb, n_orb)
* ``"d"``     d[p, q, r, s] = sum_{s1, s2} <a+_{p s1} a+_{r s2} a_{s s2} a_{q s1}>
  (n_orb,)*4, chemists' order: E = sum h_pq D_pq + 1/2 sum (pq|rs) d_pqrs
  for the Hamiltonian of the "Unitary coupled cluster" subsection, and the
  electron count is trace(D).

The rows are built on the host once per (n_so, kinds), as input preparation;
every element is then computed on the GPU, and the host only reshapes.
"""

import numpy as np

from .inputs.hamiltonian import PauliSum, fermion_monomial_map

KINDS = ("1rdm", "2rdm", "D", "d")


def _grid(n, k):
    return [a.ravel() for a in np.meshgrid(*([np.arange(n)] * k), indexing="ij")]


def rdm_rows(n_so: int, kind: str, tol: float = 1e-14):
    """(strings (T, n_so) uint8, row_ptr, cols, weights complex, shape) of one kind."""
    if n_so % 2 or n_so < 2:
        raise ValueError("n_so must be a positive even number of spin orbitals")
    n_orb = n_so // 2
    if kind == "1rdm":
        P, Q = _grid(n_so, 2)
        ops, row, shape = [(P, True), (Q, False)], np.arange(P.size), (n_so, n_so)
    elif kind == "2rdm":
        P, Q, R, S = _grid(n_so, 4)
        ops, row, shape = [(P, True), (Q, True), (R, False), (S, False)], np.arange(P.size), (n_so,) * 4
    elif kind == "D":
        p, q = _grid(n_orb, 2)
        rows = np.arange(p.size)
        ops = [(np.concatenate([2 * p + s for s in (0, 1)]), True),
               (np.concatenate([2 * q + s for s in (0, 1)]), False)]
        row, shape = np.concatenate([rows, rows]), (n_orb, n_orb)
    elif kind == "d":
        p, q, r, s = _grid(n_orb, 4)
        rows = np.arange(p.size)
        cat = lambda f: np.concatenate([f(s1, s2) for s1 in (0, 1) for s2 in (0, 1)])  # noqa: E731
        ops = [(cat(lambda s1, s2: 2 * p + s1), True), (cat(lambda s1, s2: 2 * r + s2), True),
               (cat(lambda s1, s2: 2 * s + s2), False), (cat(lambda s1, s2: 2 * q + s1), False)]
        row, shape = np.concatenate([rows] * 4), (n_orb,) * 4
    else:
        raise ValueError(f"unknown RDM kind {kind!r}; expected one of {KINDS}")
    strings, rp, cols, w = fermion_monomial_map(n_so, ops, tol)
    n_rows = int(np.prod(shape))
    # sum the monomials of each row (several for the spin-summed kinds)
    mono = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    T = max(1, strings.shape[0])
    key = row[mono].astype(np.int64) * T + cols
    ukey, inv = np.unique(key, return_inverse=True)
    ww = (np.bincount(inv, weights=w.real, minlength=ukey.size)
          + 1j * np.bincount(inv, weights=w.imag, minlength=ukey.size))
    keep = np.abs(ww) > tol
    ukey, ww = ukey[keep], ww[keep]
    r_of, c_of = ukey // T, ukey % T
    used, cols2 = np.unique(c_of, return_inverse=True)
    row_ptr = np.searchsorted(r_of, np.arange(n_rows + 1)).astype(np.int64)
    return strings[used], row_ptr, cols2.astype(np.int32), ww, shape


def merged_rows(n_so: int, kinds):
    """One string set and one row list for several kinds (rows in ``kinds``
    order).  Returns (strings, row_ptr, cols, weights, [(kind, row offset, shape)])."""
    parts = [rdm_rows(n_so, k) for k in kinds]
    allstr = np.concatenate([p[0] for p in parts]) if parts else np.zeros((0, n_so), np.uint8)
    uniq, inv = np.unique(allstr, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    row_ptr, cols, weights, layout = [np.zeros(1, np.int64)], [], [], []
    s_off, r_off, e_off = 0, 0, 0
    for k, (strings, rp, c, w, shape) in zip(kinds, parts):
        cols.append(inv[s_off + c])
        weights.append(w)
        row_ptr.append(rp[1:] + e_off)
        layout.append((k, r_off, shape))
        s_off += strings.shape[0]
        r_off += rp.size - 1
        e_off += int(rp[-1])
    return (uniq.astype(np.uint8), np.concatenate(row_ptr), np.concatenate(cols).astype(np.int32),
            np.concatenate(weights), layout)


class RDM:
    """RDM evaluator bound to a context: the string set (a Hamiltonian
    handle) and the rows (an Observables handle) are uploaded once; calling
    it on a state returns {kind: complex array} computed on the GPU."""

    def __init__(self, ctx, n_so: int, kinds=("1rdm", "2rdm")):
        from . import mps

        for k in kinds:
            if k not in KINDS:
                raise ValueError(f"unknown RDM kind {k!r}; expected one of {KINDS}")
        self.n_so = int(n_so)
        self.kinds = tuple(kinds)
        strings, row_ptr, cols, weights, self.layout = merged_rows(self.n_so, self.kinds)
        self.n_strings = int(strings.shape[0])
        self.strings = mps.Hamiltonian(ctx, PauliSum(self.n_so, strings, np.ones(self.n_strings)))
        self.obs = mps.Observables(self.strings, row_ptr, cols, weights)

    def __call__(self, state) -> dict:
        vals = state.observables(self.obs)
        return {k: vals[off: off + int(np.prod(shape))].reshape(shape).copy() for k, off, shape in self.layout}
