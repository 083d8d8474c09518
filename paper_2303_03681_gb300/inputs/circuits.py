"""Gate lists for the MPS simulator.

Conventions shared with the C-ABI:

* a two-qubit gate acts on the adjacent sites (q, q+1); its 4x4 matrix is
  indexed by 2*i_q + i_{q+1} (site q is the more significant bit);
* a one-qubit gate acts on site q and uses the top-left 2x2 block;
* a gate of a circuit *template* may depend on one variational angle:
  G = exp(i phi) M_plus + exp(-i phi) M_minus with phi = coeff * theta[param]
  (a fixed gate has param = -1 and M_minus = 0).

Circuits:

* brickwork: layer l applies Haar-random SU(4) gates on the bonds (2k, 2k+1)
  for even l and (2k+1, 2k+2) for odd l;
* UCCSD-style: the first-order Trotter product of the spin-conserving single
  and double excitations of a Hartree-Fock reference (the paper's UCCSD
  subsection), every generator theta (tau - tau^dagger) JW-mapped to
  sum_k i c_k P_k and applied as prod_k exp(i theta c_k P_k); each Pauli
  exponential is compiled to one- and two-qubit gates: a basis change on the
  support (H for X, Rx(pi/2) for Y), a nearest-neighbour parity ladder over
  [min, max] of the support (CNOT(j -> j+1) when site j+1 is in the support,
  SWAP otherwise), exp(i phi Z) on the last support site, and the mirror
  ladder.  The one-qubit basis changes and the rotation are multiplied into
  the adjacent two-qubit gates, so a string spanning sites a..b becomes
  2 (b - a) - 1 two-qubit gates, one of which carries the angle.
"""

from dataclasses import dataclass, field

import numpy as np

from .hamiltonian import fermion_terms_to_paulis

I2 = np.eye(2, dtype=complex)
HADAMARD = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2.0)
RX_HALF_PI = np.array([[1, -1j], [-1j, 1]], dtype=complex) / np.sqrt(2.0)
CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=complex)
PROJ0 = np.diag([1.0, 0.0]).astype(complex)
PROJ1 = np.diag([0.0, 1.0]).astype(complex)


@dataclass
class GateList:
    """A concrete gate sequence (applied in list order)."""

    n_qubits: int
    q: np.ndarray  # (G,) int32, first site
    arity: np.ndarray  # (G,) int32, 1 or 2
    u: np.ndarray  # (G, 4, 4) complex128

    @property
    def n_gates(self) -> int:
        return int(self.q.shape[0])

    @property
    def n_two_qubit(self) -> int:
        return int(np.count_nonzero(self.arity == 2))

    def slice(self, stop: int) -> "GateList":
        return GateList(self.n_qubits, self.q[:stop], self.arity[:stop], self.u[:stop])


@dataclass
class CircuitTemplate:
    """A gate sequence whose parametrised gates are bound from theta."""

    n_qubits: int
    n_params: int
    q: np.ndarray
    arity: np.ndarray
    param: np.ndarray  # (G,) int32, -1 for fixed gates
    coeff: np.ndarray  # (G,) float64
    m_plus: np.ndarray  # (G, 4, 4) complex128
    m_minus: np.ndarray  # (G, 4, 4) complex128
    meta: dict = field(default_factory=dict)

    @property
    def n_gates(self) -> int:
        return int(self.q.shape[0])

    @property
    def n_two_qubit(self) -> int:
        return int(np.count_nonzero(self.arity == 2))

    def bind(self, theta) -> GateList:
        theta = np.asarray(theta, dtype=float)
        if theta.shape != (self.n_params,):
            raise ValueError(f"theta has shape {theta.shape}, expected ({self.n_params},)")
        if self.n_params == 0:
            phi = np.zeros(self.n_gates)
        else:
            phi = np.where(self.param >= 0, self.coeff * theta[np.maximum(self.param, 0)], 0.0)
        u = (np.exp(1j * phi)[:, None, None] * self.m_plus
             + np.exp(-1j * phi)[:, None, None] * self.m_minus)
        return GateList(self.n_qubits, self.q.copy(), self.arity.copy(), u)

    def prefix(self, n_gates: int) -> "CircuitTemplate":
        """The first ``n_gates`` gates (the angles keep their indices)."""
        return CircuitTemplate(self.n_qubits, self.n_params, self.q[:n_gates], self.arity[:n_gates],
                               self.param[:n_gates], self.coeff[:n_gates], self.m_plus[:n_gates],
                               self.m_minus[:n_gates], dict(self.meta))

    @staticmethod
    def from_gates(gl: GateList) -> "CircuitTemplate":
        g = gl.n_gates
        return CircuitTemplate(gl.n_qubits, 0, gl.q.copy(), gl.arity.copy(), np.full(g, -1, np.int32),
                               np.zeros(g), gl.u.copy(), np.zeros_like(gl.u))


class _Builder:
    def __init__(self, n):
        self.n = n
        self.q, self.arity, self.param, self.coeff, self.mp, self.mm = [], [], [], [], [], []

    def fixed(self, q, arity, u):
        self.q.append(q)
        self.arity.append(arity)
        self.param.append(-1)
        self.coeff.append(0.0)
        self.mp.append(_pad4(u))
        self.mm.append(np.zeros((4, 4), complex))

    def rotation(self, q, arity, param, coeff, m_plus, m_minus):
        self.q.append(q)
        self.arity.append(arity)
        self.param.append(param)
        self.coeff.append(coeff)
        self.mp.append(_pad4(m_plus))
        self.mm.append(_pad4(m_minus))

    def template(self, n_params, meta=None):
        g = len(self.q)
        return CircuitTemplate(
            self.n, n_params,
            np.asarray(self.q, np.int32).reshape(g), np.asarray(self.arity, np.int32).reshape(g),
            np.asarray(self.param, np.int32).reshape(g), np.asarray(self.coeff, float).reshape(g),
            np.asarray(self.mp, complex).reshape(g, 4, 4), np.asarray(self.mm, complex).reshape(g, 4, 4),
            meta or {})


def _pad4(u):
    u = np.asarray(u, dtype=complex)
    if u.shape == (4, 4):
        return u
    out = np.zeros((4, 4), complex)
    out[:2, :2] = u
    return out


# ----------------------------------------------------------------------------
# brickwork
# ----------------------------------------------------------------------------

def haar_su4(rng: np.random.Generator) -> np.ndarray:
    """Haar-random SU(4): QR of a complex Ginibre matrix with the phases of
    R's diagonal moved into Q, then divided by a fourth root of det."""
    z = (rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))) / np.sqrt(2.0)
    qm, r = np.linalg.qr(z)
    d = np.diag(r)
    qm = qm * (d / np.abs(d))[None, :]
    det = np.linalg.det(qm)
    return qm / det ** 0.25


def brickwork_circuit(n: int, layers: int, rng: np.random.Generator) -> GateList:
    qs, us = [], []
    for layer in range(layers):
        for q in range(layer % 2, n - 1, 2):
            qs.append(q)
            us.append(haar_su4(rng))
    g = len(qs)
    return GateList(n, np.asarray(qs, np.int32), np.full(g, 2, np.int32),
                    np.asarray(us, complex).reshape(g, 4, 4))


# ----------------------------------------------------------------------------
# UCCSD-style circuits
# ----------------------------------------------------------------------------

def uccsd_excitations(n_so: int, n_electrons: int):
    """Spin-conserving singles (i -> a) then doubles (i<j -> a<b), lexicographic.

    Spin orbitals are interleaved (spin = index % 2); occupied = the lowest
    n_electrons.  Returns a list of tuples (i, a) and (i, j, a, b).
    """
    occ = list(range(n_electrons))
    vir = list(range(n_electrons, n_so))
    singles = [(i, a) for i in occ for a in vir if i % 2 == a % 2]
    doubles = []
    for ii, i in enumerate(occ):
        for j in occ[ii + 1:]:
            for aa, a in enumerate(vir):
                for b in vir[aa + 1:]:
                    if sorted((i % 2, j % 2)) == sorted((a % 2, b % 2)):
                        doubles.append((i, j, a, b))
    return singles + doubles


def excitation_generator_paulis(n_so: int, exc):
    """JW strings of tau - tau^dagger as (ops (K, n) uint8, c (K,) real) with
    tau - tau^dagger = sum_k i c_k P_k.

    tau = a+_a a_i for a single (i, a); tau = a+_a a+_b a_j a_i for a double
    (i, j, a, b).
    """
    one = np.ones(1)
    if len(exc) == 2:
        i, a = exc
        tau = [([a], True), ([i], False)]
        tau_dag = [([i], True), ([a], False)]
    else:
        i, j, a, b = exc
        tau = [([a], True), ([b], True), ([j], False), ([i], False)]
        tau_dag = [([i], True), ([j], True), ([b], False), ([a], False)]
    ops, vals = fermion_terms_to_paulis(n_so, [(one, tau), (-one, tau_dag)])
    if np.max(np.abs(vals.real), initial=0.0) > 1e-12:
        raise ValueError("excitation generator is not anti-Hermitian")
    return ops, vals.imag.copy()


def _basis_change(op: int) -> np.ndarray:
    """U with U P U^dagger = Z for P in {X, Y, Z}."""
    return {1: HADAMARD, 2: RX_HALF_PI, 3: I2}[int(op)]


def _emit_pauli_exponential(bld: _Builder, ops_row, param: int, coeff: float):
    """Append the compiled exp(i phi P), phi = coeff * theta[param]."""
    support = np.nonzero(ops_row)[0]
    if support.size == 0:
        return  # global phase
    a, b = int(support[0]), int(support[-1])
    basis = {int(s): _basis_change(ops_row[s]) for s in support}
    if a == b:
        u = basis[a]
        bld.rotation(a, 1, param, coeff, u.conj().T @ PROJ0 @ u, u.conj().T @ PROJ1 @ u)
        return
    in_support = set(basis)

    def ladder(j):
        return CNOT if (j + 1) in in_support else SWAP

    def before(j):  # basis changes applied just before the forward gate on bond j
        first = basis[a] if j == a else I2
        second = basis[j + 1] if (j + 1) in in_support else I2
        return np.kron(first, second)

    def after(j):  # inverse basis changes applied just after the mirror gate on bond j
        first = basis[a].conj().T if j == a else I2
        second = basis[j + 1].conj().T if (j + 1) in in_support else I2
        return np.kron(first, second)

    for j in range(a, b - 1):
        bld.fixed(j, 2, ladder(j) @ before(j))
    j = b - 1
    g = ladder(j)
    m_plus = after(j) @ g @ np.kron(I2, PROJ0) @ g @ before(j)
    m_minus = after(j) @ g @ np.kron(I2, PROJ1) @ g @ before(j)
    bld.rotation(j, 2, param, coeff, m_plus, m_minus)
    for j in range(b - 2, a - 1, -1):
        bld.fixed(j, 2, after(j) @ ladder(j))


def pauli_exponential_template(n: int, strings, n_params: int, meta=None) -> CircuitTemplate:
    """Template of prod_k exp(i coeff_k theta[param_k] P_k), k in list order.

    ``strings`` is an iterable of (ops_row (n,) uint8, param, coeff).
    """
    bld = _Builder(n)
    for ops_row, param, coeff in strings:
        _emit_pauli_exponential(bld, np.asarray(ops_row), int(param), float(coeff))
    return bld.template(n_params, meta)


def uccsd_template(n_so: int, n_electrons: int, max_excitations=None) -> CircuitTemplate:
    """UCCSD-style template: one angle per excitation, strings in generator order.

    ``max_excitations`` keeps only the first that many excitations (singles
    come first); None keeps them all.
    """
    excs = uccsd_excitations(n_so, n_electrons)
    if max_excitations is not None:
        excs = excs[:max_excitations]
    strings = []
    n_strings = 0
    for k, exc in enumerate(excs):
        ops, c = excitation_generator_paulis(n_so, exc)
        for row, ck in zip(ops, c):
            strings.append((row, k, ck))
            n_strings += 1
    meta = {"n_excitations": len(excs), "n_pauli_exponentials": n_strings}
    return pauli_exponential_template(n_so, strings, len(excs), meta)


# ----------------------------------------------------------------------------
# windowed generalised-singles-and-doubles pool (hydrogen-chain ansatz)
# ----------------------------------------------------------------------------

def gsd_excitations(orbitals):
    """Spin-conserving generalised singles and doubles among the spatial
    ``orbitals`` (every spin orbital may be created or annihilated, no
    occupied/virtual split).  Tuples in the convention of
    ``excitation_generator_paulis``: (i, a) for tau = a+_a a_i and
    (i, j, a, b) for tau = a+_a a+_b a_j a_i; each pair {tau, tau^dagger}
    appears once."""
    so = sorted(2 * p + s for p in orbitals for s in (0, 1))
    singles = [(q, p) for p in so for q in so if p > q and p % 2 == q % 2]
    pairs = [(p, q) for p in so for q in so if p > q]
    doubles = []
    for a, b in pairs:  # created: a > b
        for j, i in pairs:  # annihilated: j > i
            if (a, b) > (j, i) and sorted((a % 2, b % 2)) == sorted((i % 2, j % 2)):
                doubles.append((i, j, a, b))
    return singles + doubles


def windowed_gsd_pool(n_orb: int, window: int = 5) -> np.ndarray:
    """Operator pool of the paper's hydrogen-chain ansatz (Methods, "The wave
    function ansatz for hydrogen chain simulations"): generalised singles and
    doubles within every run of ``window`` consecutive spatial orbitals, each
    generator JW-mapped to Pauli strings, every Z replaced by I, strings with
    an even number of Y dropped, duplicates removed.

    Returns the distinct strings as (K, 2 n_orb) uint8, lexicographically
    sorted; each enters a circuit as exp(i theta P)."""
    n_so = 2 * n_orb
    w = min(window, n_orb)
    seen = set()
    rows = []
    for start in range(0, n_orb - w + 1):
        for exc in gsd_excitations(range(start, start + w)):
            ops, _ = excitation_generator_paulis(n_so, exc)
            for row in ops:
                r = np.where(row == 3, 0, row).astype(np.uint8)
                if not r.any() or np.count_nonzero(r == 2) % 2 == 0:
                    continue
                key = r.tobytes()
                if key not in seen:
                    seen.add(key)
                    rows.append(r)
    if not rows:
        return np.zeros((0, n_so), np.uint8)
    out = np.array(rows, dtype=np.uint8)
    return out[np.lexsort(out.T[::-1])]


def pauli_product_template(n: int, pool: np.ndarray, chosen) -> CircuitTemplate:
    """prod_k exp(i theta[k] pool[chosen[k]]) in order, one angle per factor
    (the adaptive circuit of the hydrogen-chain ansatz)."""
    strings = [(pool[j], k, 1.0) for k, j in enumerate(chosen)]
    return pauli_exponential_template(n, strings, len(strings), {"chosen": list(map(int, chosen))})
