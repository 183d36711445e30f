"""Seeded synthetic workloads: problem descriptions and random inputs.

This module is the only code shared by the CUDA path's tests/benchmarks and the CPU oracle.
It holds none of the method's arithmetic: it describes a problem by its raw physical
parameters (the numbers a user would type into a config) and draws random control vectors
and window states from a counter-based generator.  Everything derived from the
parameters (drift energies, ladder operators, spline placement, targets, time grid) is
computed separately by each side.

Random numbers come from splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used as a counter-based generator: element ``j`` of a
stream keyed by ``(seed, problem, tensor)`` is ``mix64(key + (j + 1) * GOLDEN)``.  The same
seed therefore always gives the same array on any machine.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

TWO_PI = 2.0 * math.pi

# tensor ids for the counter-based streams
STREAM_ALPHA = 1
STREAM_W_RE = 2
STREAM_W_IM = 3
STREAM_MISC = 4


def _mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, problem: int, tensor: int) -> np.uint64:
    """Key of one random stream (seed, problem index, tensor id)."""
    with np.errstate(over="ignore"):
        k = _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + GOLDEN)
        k = _mix64(k ^ (np.uint64(problem & 0xFFFFFFFF) * _M1 + GOLDEN))
        k = _mix64(k ^ (np.uint64(tensor & 0xFFFFFFFF) * _M2 + GOLDEN))
    return np.uint64(k)


def uniform01(seed: int, problem: int, tensor: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from stream (seed, problem, tensor); 53 random bits each."""
    key = stream_key(seed, problem, tensor)
    j = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix64(key + j * GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, problem: int, tensor: int, n: int, lo: float, hi: float) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, problem, tensor, n)


@dataclasses.dataclass
class ProblemSpec:
    """Raw description of one multiple-shooting problem.

    q subsystems with L levels each, of which the lowest ``ness`` are essential; the state
    matrix is N x E with N = L**q and E = ness**q.  Drift parameters are given in rad/ns:
    ``xi[k]`` self-Kerr, ``xi_cross[k][l]`` cross-Kerr (k < l used), and optionally the
    paper's own model: ``detune[k]`` (omega_k - omega_rot) and ``jx[k][l]`` dipole exchange.
    ``omega[k]`` lists the carrier frequencies of subsystem k (rad/ns); each carrier has
    ``d1`` B-spline coefficients (complex, i.e. two reals).  ``T`` is the gate duration in
    ns, ``nsteps`` the global number of time steps and ``M`` the number of windows.
    ``mu`` <= 0 selects the default penalty weight.
    """

    q: int
    L: int
    ness: int
    xi: List[float]
    xi_cross: List[List[float]]
    omega: List[List[float]]
    d1: int
    T: float
    nsteps: int
    M: int
    mu: float = 0.0
    detune: Optional[List[float]] = None
    jx: Optional[List[List[float]]] = None
    name: str = ""

    @property
    def N(self) -> int:
        return self.L ** self.q

    @property
    def E(self) -> int:
        return self.ness ** self.q

    @property
    def nf(self) -> List[int]:
        return [len(w) for w in self.omega]

    @property
    def d(self) -> int:
        """Number of real control parameters: two per spline coefficient."""
        return 2 * self.d1 * sum(self.nf)

    @property
    def nW(self) -> int:
        """Number of doubles in the window-state vector W^1..W^{M-1} (complex interleaved)."""
        return 2 * self.N * self.E * (self.M - 1)

    def replace(self, **kw) -> "ProblemSpec":
        return dataclasses.replace(self, **kw)


def transmon_spec(q: int, T: float, nsteps: int, M: int, d1: int, *, L: int = 3, ness: int = 2,
                  xi_ghz: float = 0.22, xi_cross_ghz: float = 0.001, name: str = "") -> ProblemSpec:
    """q transmons, L levels (ness essential), all-pair cross-Kerr, carriers {0, -xi_k}.

    Frequencies are given in GHz and converted to rad/ns (factor 2*pi).
    """
    xi = [TWO_PI * xi_ghz] * q
    xc = [[(TWO_PI * xi_cross_ghz if l > k else 0.0) for l in range(q)] for k in range(q)]
    omega = [[0.0, -xi[k]] for k in range(q)]
    return ProblemSpec(q=q, L=L, ness=ness, xi=xi, xi_cross=xc, omega=omega, d1=d1, T=T,
                       nsteps=nsteps, M=M, name=name or f"{q}q")


# The workloads: 2-, 3-, 4- and 5-transmon shapes of the QFT benchmarks.
def config_2q(M: int = 8) -> ProblemSpec:
    return transmon_spec(2, 100.0, 4000, M, 10, name="2q-N9-E4")


def config_3q(M: int = 32) -> ProblemSpec:
    return transmon_spec(3, 300.0, 20000, M, 20, name="3q-N27-E8")


def config_4q(M: int = 64) -> ProblemSpec:
    return transmon_spec(4, 600.0, 100000, M, 40, name="4q-N81-E16")


def config_5q(M: int = 256) -> ProblemSpec:
    return transmon_spec(5, 800.0, 150000, M, 53, name="5q-N243-E32")


# The paper's own test cases (Table 1): q qubits (2 levels, all essential) in a linear chain,
# rotating frame at the mean transition frequency, dipole exchange between neighbours, the
# listed carrier frequencies, B-spline spacing 3 ns; durations and step counts of Table 2.
PAPER_OMEGA_GHZ = [5.18, 5.12, 5.06, 5.0]
PAPER_J_GHZ = 0.005
PAPER_CARRIERS_MHZ = {
    2: [[-30.41, 30.41], [-30.41, 30.41]],
    3: [[0.0, -60.4], [60.4, 0.0, -60.4], [60.4, 0.0]],
    4: [[-30.0, -90.41], [30.0, -30.0, -90.41], [90.41, 30.0, -30.0], [90.41, -30.0]],
}
PAPER_T_NS = {2: 190.0, 3: 500.0, 4: 900.0}
PAPER_NSTEPS = {2: 2252, 3: 19806, 4: 106072}


def paper_qft_spec(q: int, M: int = 1, nsteps: Optional[int] = None) -> ProblemSpec:
    """QFT-2^q on q qubits with the paper's system parameters (Table 1) and time grid (Table 2).
    nsteps, if given, replaces the table's step count with the same duration."""
    om = PAPER_OMEGA_GHZ[:q]
    rot = sum(om) / q
    detune = [TWO_PI * (w - rot) for w in om]
    jx = [[(TWO_PI * PAPER_J_GHZ if l == k + 1 else 0.0) for l in range(q)] for k in range(q)]
    omega = [[TWO_PI * f * 1e-3 for f in fs] for fs in PAPER_CARRIERS_MHZ[q]]
    T = PAPER_T_NS[q]
    d1 = int(math.ceil(T / 3.0)) + 2
    return ProblemSpec(q=q, L=2, ness=2, xi=[0.0] * q, xi_cross=[[0.0] * q for _ in range(q)], omega=omega,
                       d1=d1, T=T, nsteps=nsteps or PAPER_NSTEPS[q], M=M, detune=detune, jx=jx,
                       name=f"QFT-{2 ** q}")


ALPHA_AMP = TWO_PI * 0.004  # rad/ns: control coefficients are uniform in +-ALPHA_AMP
PAPER_ALPHA0_AMP = TWO_PI * 0.010  # rad/ns: the paper's initial guess, uniform in +-10 MHz (Sec. 5)


def random_alpha(spec: ProblemSpec, seed: int, problem: int = 0, amp: float = ALPHA_AMP) -> np.ndarray:
    """Control vector, layout [k][f][s][re, im], iid uniform in [-amp, amp]."""
    return uniform(seed, problem, STREAM_ALPHA, spec.d, -amp, amp)


def random_W(spec: ProblemSpec, seed: int, problem: int = 0) -> np.ndarray:
    """Window states W^1..W^{M-1}: [M-1][E][N] complex interleaved as doubles.

    Real and imaginary parts iid uniform in [-a, a] with a = sqrt(3 / (2 N)), so that each
    column has unit expected squared norm.
    """
    n = spec.N * spec.E * (spec.M - 1)
    a = math.sqrt(3.0 / (2.0 * spec.N))
    re = uniform(seed, problem, STREAM_W_RE, n, -a, a)
    im = uniform(seed, problem, STREAM_W_IM, n, -a, a)
    out = np.empty(2 * n, dtype=np.float64)
    out[0::2] = re
    out[1::2] = im
    return out


def perturbed_duration_spec(base: ProblemSpec, factor: float, M: int) -> ProblemSpec:
    """Same system with duration factor*T; the step size is kept: nsteps scales with T."""
    return base.replace(T=base.T * factor, nsteps=int(round(base.nsteps * factor)), M=M,
                        name=f"{base.name}-x{factor:.3f}-M{M}")


def mixed_batch_specs(seed: int, n_per_shape: int, shapes: Sequence[ProblemSpec],
                      window_choices: Sequence[int] = (8, 32, 64, 128)) -> List[ProblemSpec]:
    """Batched workload: n_per_shape problems of each shape, durations uniform in
    [0.5 T, 1.5 T] (step size kept), window counts drawn from window_choices."""
    specs: List[ProblemSpec] = []
    u = uniform01(seed, 0, STREAM_MISC, 2 * n_per_shape * len(shapes))
    idx = 0
    for base in shapes:
        for _ in range(n_per_shape):
            factor = 0.5 + u[idx]
            M = int(window_choices[min(int(u[idx + 1] * len(window_choices)), len(window_choices) - 1)])
            idx += 2
            sp = perturbed_duration_spec(base, factor, M)
            specs.append(sp)
    return specs
