"""The variational loop around the energy evaluations (UCC, Eq. ucc).

VQE minimises E(theta) = <psi(theta)|H|psi(theta)> over the angles of the
UCCSD-style circuit.  The paper optimises with BOBYQA, a derivative-free
trust-region method (Results, H2 potential-energy curves).  This module keeps
the loop derivative-free but shapes it for a batched evaluator: every step
asks for a block of independent energies at once, which the GPU evaluates
concurrently (one state and stream per slot, ``vqe_eval_batch``), or which a
``Server`` runs alongside other clients' requests.

Both optimisers rest on one property of the circuits built by
``inputs.uccsd_template``: the Pauli exponentials of one excitation commute,
so together they are exactly exp(theta_k G_k) with G_k = tau_k - tau_k^dagger,
and a single or double excitation generator satisfies G^3 = -G.  Hence
exp(s G) = 1 + sin(s) G + (1 - cos(s)) G^2, and with the other angles fixed

    E(theta_k + s) = a0 + a1 cos s + b1 sin s + a2 cos 2s + b2 sin 2s.

* ``sequential_minimize``: per angle, 4 new energies at s = 2 pi j / 5
  (j = 1..4; j = 0 is the current point) fix the five coefficients, and the
  angle moves to the exact minimum of that trigonometric polynomial
  (sequential minimal optimisation, Nakanishi, Fujii and Todo, Phys. Rev.
  Research 2, 043158 (2020), for this frequency set).
* ``shift_gradient``: E'(theta_k) = D2 + (1 - sqrt 2) D1 / 2 with
  D1 = E(+pi/2) - E(-pi/2) and D2 = E(+pi/4) - E(-pi/4), 4 energies per angle,
  all angles in one batch; ``bfgs_minimize`` uses it with a batched
  backtracking line search (all trial steps in one batch).

Under bond-dimension truncation the expansion holds only up to the discarded
weight; the optimisers re-evaluate the energy after every sweep or step, so
their reported energies are always measured ones.

The optimisers take any ``energy_batch(thetas (B, P)) -> energies (B,)``;
``BatchedEnergy`` and ``ServedEnergy`` supply it from the CUDA library.
"""

from dataclasses import dataclass, field

import numpy as np

_FIVE = 2.0 * np.pi * np.arange(5) / 5.0


# ---------------------------------------------------------------------------
# one angle: the degree-2 trigonometric model
# ---------------------------------------------------------------------------

def trig_coefficients(e5) -> np.ndarray:
    """(a0, a1, b1, a2, b2) of the degree-2 trigonometric polynomial through
    the five values e5[j] = E(2 pi j / 5) (exact for such polynomials)."""
    e5 = np.asarray(e5, dtype=float)
    if e5.shape != (5,):
        raise ValueError("need the energies at the five shifts 2 pi j / 5")
    c1, s1 = np.cos(_FIVE), np.sin(_FIVE)
    c2, s2 = np.cos(2 * _FIVE), np.sin(2 * _FIVE)
    return np.array([e5.mean(), 0.4 * e5 @ c1, 0.4 * e5 @ s1, 0.4 * e5 @ c2, 0.4 * e5 @ s2])


def trig_value(coef, s):
    a0, a1, b1, a2, b2 = coef
    s = np.asarray(s, dtype=float)
    return a0 + a1 * np.cos(s) + b1 * np.sin(s) + a2 * np.cos(2 * s) + b2 * np.sin(2 * s)


def trig_argmin(coef) -> float:
    """Global minimiser in (-pi, pi] of the degree-2 trigonometric polynomial.

    Candidates are the stationary points (the roots z = e^{is} of the quartic
    that E'(s) = 0 becomes after multiplying by 2 i z^2) and the best point
    of a uniform grid; each is polished with Newton steps on E'."""
    a0, a1, b1, a2, b2 = (float(c) for c in coef)
    quartic = np.array([-2 * a2 + 2j * b2, -a1 + 1j * b1, 0.0, a1 + 1j * b1, 2 * a2 + 2j * b2])
    cands = []
    if np.any(np.abs(quartic) > 0):
        nz = np.nonzero(np.abs(quartic) > 1e-300)[0]
        if nz.size and nz[0] < 4:
            cands += list(np.angle(np.roots(quartic[nz[0]:])))
    grid = np.linspace(-np.pi, np.pi, 256, endpoint=False)
    cands.append(float(grid[np.argmin(trig_value(coef, grid))]))
    best_s, best_e = 0.0, float(trig_value(coef, 0.0))
    for s in cands:
        s = float(s)
        for _ in range(30):
            d1 = -a1 * np.sin(s) + b1 * np.cos(s) - 2 * a2 * np.sin(2 * s) + 2 * b2 * np.cos(2 * s)
            d2 = -a1 * np.cos(s) - b1 * np.sin(s) - 4 * a2 * np.cos(2 * s) - 4 * b2 * np.sin(2 * s)
            if d2 <= 0:
                break
            step = d1 / d2
            s -= step
            if abs(step) < 1e-15:
                break
        e = float(trig_value(coef, s))
        if e < best_e:
            best_s, best_e = s, e
    return float(np.angle(np.exp(1j * best_s)))  # wrapped to (-pi, pi]


# ---------------------------------------------------------------------------
# optimisers
# ---------------------------------------------------------------------------

@dataclass
class VqeResult:
    theta: np.ndarray
    energy: float  # a measured energy at theta (never a model value)
    converged: bool
    iterations: int  # sweeps (sequential) or steps (BFGS)
    n_evals: int  # energies requested from the evaluator
    n_batches: int  # evaluator calls
    history: list = field(default_factory=list)  # measured energy after each sweep / step


class _Counter:
    def __init__(self, energy_batch):
        self.f = energy_batch
        self.n_evals = 0
        self.n_batches = 0

    def __call__(self, thetas):
        thetas = np.atleast_2d(np.asarray(thetas, dtype=float))
        out = np.asarray(self.f(thetas), dtype=float).reshape(-1)
        if out.shape[0] != thetas.shape[0]:
            raise ValueError("energy_batch returned the wrong number of energies")
        self.n_evals += thetas.shape[0]
        self.n_batches += 1
        return out


def sequential_minimize(energy_batch, theta0, max_sweeps: int = 20, tol: float = 1e-10,
                        order=None) -> VqeResult:
    """Exact coordinate-wise minimisation, one angle at a time in ``order``
    (default 0..P-1), each step one batch of 4 energies.  Stops when a sweep
    lowers the measured energy by less than ``tol`` (or after max_sweeps)."""
    f = _Counter(energy_batch)
    theta = np.array(theta0, dtype=float)
    P = theta.shape[0]
    order = np.arange(P) if order is None else np.asarray(order)
    e = float(f(theta[None])[0])
    hist = [e]
    converged = False
    sweeps = 0
    for sweeps in range(1, max_sweeps + 1):
        for k in order:
            trial = np.repeat(theta[None], 4, axis=0)
            trial[:, k] += _FIVE[1:]
            e5 = np.concatenate([[e], f(trial)])
            coef = trig_coefficients(e5)
            s = trig_argmin(coef)
            theta[k] = float(np.angle(np.exp(1j * (theta[k] + s))))
            e = float(trig_value(coef, s))
        e = float(f(theta[None])[0])  # the measured energy replaces the model's
        hist.append(e)
        if hist[-2] - hist[-1] < tol:
            converged = True
            break
    return VqeResult(theta, e, converged, sweeps, f.n_evals, f.n_batches, hist)


def shift_gradient(energy_batch, theta) -> np.ndarray:
    """Exact gradient from 4 shifted energies per angle, all in one batch."""
    theta = np.asarray(theta, dtype=float)
    P = theta.shape[0]
    shifts = np.array([np.pi / 2, -np.pi / 2, np.pi / 4, -np.pi / 4])
    trial = np.repeat(theta[None], 4 * P, axis=0)
    for k in range(P):
        trial[4 * k: 4 * k + 4, k] += shifts
    e = np.asarray(energy_batch(trial), dtype=float).reshape(P, 4)
    d1 = e[:, 0] - e[:, 1]
    d2 = e[:, 2] - e[:, 3]
    return d2 + (1.0 - np.sqrt(2.0)) * 0.5 * d1


def bfgs_minimize(energy_batch, theta0, max_steps: int = 100, gtol: float = 1e-7, n_trial: int = 6,
                  c1: float = 1e-4) -> VqeResult:
    """Quasi-Newton minimisation with shift-rule gradients.  The line search
    evaluates the steps 1, 1/2, ..., 2^-(n_trial-1) in one batch and takes the
    longest one with sufficient decrease (Armijo, c1)."""
    f = _Counter(energy_batch)
    x = np.array(theta0, dtype=float)
    P = x.shape[0]
    e = float(f(x[None])[0])
    g = shift_gradient(f, x)
    Hinv = np.eye(P)
    hist = [e]
    converged = False
    steps = 0
    alphas = 0.5 ** np.arange(n_trial)
    for steps in range(1, max_steps + 1):
        if np.max(np.abs(g)) < gtol:
            converged = True
            break
        p = -Hinv @ g
        slope = float(g @ p)
        if slope >= 0:  # not a descent direction: restart from steepest descent
            Hinv = np.eye(P)
            p = -g
            slope = float(g @ p)
        es = f(x[None] + alphas[:, None] * p[None])
        ok = np.nonzero(es <= e + c1 * alphas * slope)[0]
        if ok.size:
            i = int(ok[0])
        else:
            i = int(np.argmin(es))
            if es[i] >= e:
                converged = np.max(np.abs(g)) < 10 * gtol
                break
        x_new = x + alphas[i] * p
        e_new = float(es[i])
        g_new = shift_gradient(f, x_new)
        s = x_new - x
        y = g_new - g
        sy = float(s @ y)
        if sy > 1e-14 * max(1.0, float(np.linalg.norm(s) * np.linalg.norm(y))):
            rho = 1.0 / sy
            V = np.eye(P) - rho * np.outer(s, y)
            Hinv = V @ Hinv @ V.T + rho * np.outer(s, s)
        x, e, g = x_new, e_new, g_new
        hist.append(e)
    return VqeResult(x, e, converged, steps, f.n_evals, f.n_batches, hist)


# ---------------------------------------------------------------------------
# evaluators backed by the CUDA library
# ---------------------------------------------------------------------------

class BatchedEnergy:
    """energy_batch on the GPU: ``slots`` states, each on its own context and
    stream, evaluated together with vqe_eval_batch (chunks of ``slots``).

    ``state_kwargs`` go to ``mps.State`` (chi_max, precision, trunc_rel,
    svd_fp64, tensor_cores, ...)."""

    def __init__(self, template, hamiltonian, init_bits=None, slots: int = 4, device: int = 0, **state_kwargs):
        from . import mps

        self._mps = mps
        self.n_params = int(template.n_params)
        self.bits = None if init_bits is None else np.ascontiguousarray(init_bits, dtype=np.uint8)
        self.ctxs = [mps.Context(device) for _ in range(int(slots))]
        self.circuit = mps.Circuit(self.ctxs[0], template)
        self.ham = mps.Hamiltonian(self.ctxs[0], hamiltonian)
        self.states = [mps.State(c, template.n_qubits, self.bits, **state_kwargs) for c in self.ctxs]

    def __call__(self, thetas) -> np.ndarray:
        mps = self._mps
        thetas = np.atleast_2d(np.asarray(thetas, dtype=float))
        if thetas.shape[1] != self.n_params:
            raise ValueError(f"thetas have {thetas.shape[1]} angles, the circuit takes {self.n_params}")
        out = np.empty(thetas.shape[0])
        S = len(self.states)
        for lo in range(0, thetas.shape[0], S):
            chunk = thetas[lo: lo + S]
            reqs = [(st, self.circuit, self.ham, th, self.bits) for st, th in zip(self.states, chunk)]
            e, status = mps.vqe_eval_batch(reqs)
            bad = np.nonzero(status != mps.MPS_OK)[0]
            if bad.size:
                raise mps.MpsError(int(status[bad[0]]), f"evaluation {lo + int(bad[0])} of the batch failed")
            out[lo: lo + chunk.shape[0]] = e
        return out

    def close(self):
        for c in self.ctxs:
            c.close()


class ServedEnergy:
    """energy_batch through a continuous-batching ``mps.Server``: every theta
    is submitted as a request for one fragment and the results are polled in
    order.  The server may be shared with other clients; pass an existing one
    or let this object create it (``max_slots`` concurrent evaluations)."""

    def __init__(self, template, hamiltonian, init_bits=None, server=None, max_slots: int = 4, device: int = 0,
                 **fragment_kwargs):
        from . import mps

        self._mps = mps
        self.n_params = int(template.n_params)
        self._own = server is None
        self.server = mps.Server(device, max_slots) if server is None else server
        self.ctx = mps.Context(device)
        self.circuit = mps.Circuit(self.ctx, template)
        self.ham = mps.Hamiltonian(self.ctx, hamiltonian)
        self.fragment = self.server.add_fragment(self.circuit, self.ham, init_bits, **fragment_kwargs)
        self.latencies_ms = []

    def __call__(self, thetas) -> np.ndarray:
        thetas = np.atleast_2d(np.asarray(thetas, dtype=float))
        if thetas.shape[1] != self.n_params:
            raise ValueError(f"thetas have {thetas.shape[1]} angles, the circuit takes {self.n_params}")
        tickets = [self.server.submit(self.fragment, th) for th in thetas]
        out = np.empty(len(tickets))
        for i, t in enumerate(tickets):
            e, lat = self.server.poll(t, -1)
            out[i] = e
            self.latencies_ms.append(lat)
        return out

    def close(self):
        if self._own:
            self.server.close()
