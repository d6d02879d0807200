"""Seeded synthetic inputs shaped like the paper's convection / CDR workloads.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic.  Both the FP64 oracle (through the tests) and the CUDA
library are fed from it, so they see bit-identical inputs.

Recipe (all draws from ``numpy.random.Generator(PCG64(seed))`` in FP64):

* network with ``L`` hidden layers of width ``M`` and rank ``r``: ``L+1`` weight
  layers with ranks ``(r1, r, ..., r, 1)``, ``r1 = min(r, 2)`` unless given.
  ``U^l`` is ``M_l x r_l`` and ``V^l`` is ``M_{l-1} x r_l`` (``M_0 = 2`` inputs
  ``(x, t)``, ``M_{L+1} = 1`` output); entries ``N(0, 1/M)`` where the second
  argument is the variance.  Biases ``b^l ~ N(0, 0.1)`` (variance).
* coefficients ``s ~ U(0.5, 1.5)``, one vector of length ``sum(r)`` per PDE
  instance, stored layer-major.
* interior points ``(x, t) ~ U([0, 2pi] x [0, 1])``; initial points
  ``x ~ U[0, 2pi]`` at ``t = 0``; periodic pairs ``t ~ U[0, 1]`` (each pair is the
  two points ``(0, t)`` and ``(2pi, t)``).
* batched instances: ``beta ~ U[1, 20]``, ``nu ~ U[0, 5]``, ``rho ~ U[0, 5]``;
  per-instance point count log-uniform in ``[n_lo, n_hi]``, split 15/16
  interior, 1/32 initial, 1/64 periodic pairs.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

TWO_PI = 2.0 * math.pi


@dataclasses.dataclass
class Net:
    """Frozen bases of an LRNR: ``U[l]``, ``V[l]``, ``b[l]`` for the L+1 weight layers."""
    L: int                 # hidden (activated) layers
    M: int                 # hidden width
    r: list                # ranks, length L+1
    U: list                # U[l]: (M_l, r_l) float64
    V: list                # V[l]: (M_{l-1}, r_l) float64
    b: list                # b[l]: (M_l,) float64

    @property
    def sum_r(self) -> int:
        return int(sum(self.r))

    @property
    def sum_m(self) -> int:
        return self.L * self.M + 1


@dataclasses.dataclass
class Batch:
    """Instances (PDE parameter sets) and their collocation points, CSR by instance."""
    beta: np.ndarray       # (n_inst,)
    nu: np.ndarray
    rho: np.ndarray
    s: np.ndarray          # (n_inst, sum_r)
    int_off: np.ndarray    # (n_inst+1,) int64
    ic_off: np.ndarray
    bc_off: np.ndarray
    x_int: np.ndarray      # (n_int,)
    t_int: np.ndarray
    x_ic: np.ndarray       # (n_ic,)
    t_bc: np.ndarray       # (n_bc,) one entry per periodic pair

    @property
    def n_inst(self) -> int:
        return int(self.beta.shape[0])

    @property
    def n_points(self) -> int:
        """Collocation points: interior + initial + both points of each pair."""
        return int(self.x_int.shape[0] + self.x_ic.shape[0] + 2 * self.t_bc.shape[0])

    def instance(self, i: int) -> dict:
        a, b = int(self.int_off[i]), int(self.int_off[i + 1])
        c, d = int(self.ic_off[i]), int(self.ic_off[i + 1])
        e, f = int(self.bc_off[i]), int(self.bc_off[i + 1])
        return dict(beta=float(self.beta[i]), nu=float(self.nu[i]), rho=float(self.rho[i]),
                    s=self.s[i], x_int=self.x_int[a:b], t_int=self.t_int[a:b],
                    x_ic=self.x_ic[c:d], t_bc=self.t_bc[e:f])


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def ranks(L: int, r: int, r1: int | None = None) -> list:
    r1 = min(r, 2) if r1 is None else r1
    return [r1] + [r] * (L - 1) + [1]


def make_net(g: np.random.Generator, L: int, M: int, r: int, r1: int | None = None) -> Net:
    rk = ranks(L, r, r1)
    widths = [2] + [M] * L + [1]
    sd = 1.0 / math.sqrt(M)
    U, V, b = [], [], []
    for l in range(L + 1):
        U.append(g.normal(0.0, sd, size=(widths[l + 1], rk[l])))
        V.append(g.normal(0.0, sd, size=(widths[l], rk[l])))
        b.append(g.normal(0.0, math.sqrt(0.1), size=(widths[l + 1],)))
    return Net(L=L, M=M, r=rk, U=U, V=V, b=b)


def make_net_ranks(g: np.random.Generator, M: int, rk) -> Net:
    """Random bases with explicit ranks ``rk`` (L+1 entries, input layer first),
    drawn so that each layer's product U diag(s) V^T preserves the variance of its
    input: V ~ N(0, 1/M_in) (fan-in of V^T z) and U ~ N(0, 1/r_l) (fan-in of U p);
    b ~ N(0, 0.1).  (With U and V both N(0, 1/M), a wide network with rank-5 layers
    is close to a constant function: its derivative jets shrink by about r/M per
    layer and the PDE residual vanishes.)"""
    rk = [int(v) for v in rk]
    L = len(rk) - 1
    widths = [2] + [M] * L + [1]
    U, V, b = [], [], []
    for l in range(L + 1):
        U.append(g.normal(0.0, 1.0 / math.sqrt(rk[l]), size=(widths[l + 1], rk[l])))
        V.append(g.normal(0.0, 1.0 / math.sqrt(widths[l]), size=(widths[l], rk[l])))
        b.append(g.normal(0.0, math.sqrt(0.1), size=(widths[l + 1],)))
    return Net(L=L, M=M, r=rk, U=U, V=V, b=b)


def make_s(g: np.random.Generator, n_inst: int, sum_r: int) -> np.ndarray:
    return g.uniform(0.5, 1.5, size=(n_inst, sum_r))


def _offsets(counts) -> np.ndarray:
    off = np.zeros(len(counts) + 1, dtype=np.int64)
    off[1:] = np.cumsum(np.asarray(counts, dtype=np.int64))
    return off


def make_batch(g: np.random.Generator, net: Net, n_int, n_ic, n_bc, beta, nu, rho,
               s: np.ndarray | None = None) -> Batch:
    """Batch with per-instance counts ``n_int[i]``, ``n_ic[i]``, ``n_bc[i]`` (pairs)."""
    n_int, n_ic, n_bc = (np.atleast_1d(np.asarray(v, dtype=np.int64)) for v in (n_int, n_ic, n_bc))
    beta, nu, rho = (np.atleast_1d(np.asarray(v, dtype=np.float64)) for v in (beta, nu, rho))
    n_inst = beta.shape[0]
    if s is None:
        s = make_s(g, n_inst, net.sum_r)
    NI, NC, NB = int(n_int.sum()), int(n_ic.sum()), int(n_bc.sum())
    x_int = g.uniform(0.0, TWO_PI, size=NI)
    t_int = g.uniform(0.0, 1.0, size=NI)
    x_ic = g.uniform(0.0, TWO_PI, size=NC)
    t_bc = g.uniform(0.0, 1.0, size=NB)
    return Batch(beta=beta, nu=nu, rho=rho, s=np.asarray(s, dtype=np.float64),
                 int_off=_offsets(n_int), ic_off=_offsets(n_ic), bc_off=_offsets(n_bc),
                 x_int=x_int, t_int=t_int, x_ic=x_ic, t_bc=t_bc)


def make_instances(g: np.random.Generator, net: Net, n_inst: int, n_lo: int, n_hi: int,
                   fixed_count: int | None = None) -> Batch:
    """Batched CDR instances: beta~U[1,20], nu~U[0,5], rho~U[0,5]; log-uniform counts."""
    beta = g.uniform(1.0, 20.0, size=n_inst)
    nu = g.uniform(0.0, 5.0, size=n_inst)
    rho = g.uniform(0.0, 5.0, size=n_inst)
    if fixed_count is None:
        tot = np.exp(g.uniform(math.log(n_lo), math.log(n_hi), size=n_inst)).astype(np.int64)
    else:
        tot = np.full(n_inst, int(fixed_count), dtype=np.int64)
    n_int = tot * 15 // 16
    n_ic = tot // 32
    n_bc = tot // 64
    return make_batch(g, net, n_int, n_ic, n_bc, beta, nu, rho)


# ---------------------------------------------------------------------------
# The five workloads.  Seed = 1000 + workload index.
# ---------------------------------------------------------------------------

def workload_convection_small(scale: float = 1.0):
    """M=64, r=8, L=4, beta=5 (pure convection); 1,024 interior, 256 initial, 128 pairs."""
    g = rng(1000)
    net = make_net(g, L=4, M=64, r=8)
    n = lambda v: max(1, int(round(v * scale)))
    bt = make_batch(g, net, n(1024), n(256), n(128), 5.0, 0.0, 0.0)
    return net, bt


def workload_cdr_single(scale: float = 1.0):
    """M=256, r=16, L=5, CDR beta=5 nu=1 rho=2; 65,536 interior + 2,048 initial + 1,024 pairs."""
    g = rng(1001)
    net = make_net(g, L=5, M=256, r=16)
    n = lambda v: max(1, int(round(v * scale)))
    bt = make_batch(g, net, n(65536), n(2048), n(1024), 5.0, 1.0, 2.0)
    return net, bt


def workload_batched(n_inst: int = 512, n_lo: int = 1024, n_hi: int = 65536):
    """512 CDR instances, per-instance s, counts log-uniform in [1,024, 65,536]; M=256 r=16 L=5."""
    g = rng(1002)
    net = make_net(g, L=5, M=256, r=16)
    bt = make_instances(g, net, n_inst, n_lo, n_hi)
    return net, bt


def workload_adjoint_stress(n_int: int = 262144):
    """M=1,024, r=32, L=6, CDR (beta=5, nu=1, rho=2); 262,144 interior points."""
    g = rng(1003)
    net = make_net(g, L=6, M=1024, r=32)
    bt = make_batch(g, net, n_int, 0, 0, 5.0, 1.0, 2.0)
    return net, bt


def workload_spinprop(n_inst: int = 1024, per_inst: int = 16384):
    """1,024 CDR instances, 16,384 points each; M=512, r=16, L=5 (FastLRNR r_hat=16)."""
    g = rng(1004)
    net = make_net(g, L=5, M=512, r=16)
    bt = make_instances(g, net, n_inst, per_inst, per_inst, fixed_count=per_inst)
    return net, bt


def _paper_workload(seed: int, M: int, rk, mu, n_tune: int):
    g = rng(seed)
    net = make_net_ranks(g, M, rk)
    s = make_s(g, 1, net.sum_r)
    gx = TWO_PI * (np.arange(4) + 0.5) / 4.0
    gt = (np.arange(3) + 0.5) / 3.0
    X, T = np.meshgrid(gx, gt, indexing="ij")
    beta, nu, rho = mu
    bx = Batch(beta=np.array([beta]), nu=np.array([nu]), rho=np.array([rho]), s=s.copy(),
               int_off=_offsets([12]), ic_off=_offsets([0]), bc_off=_offsets([0]),
               x_int=X.ravel(), t_int=T.ravel(), x_ic=np.zeros(0), t_bc=np.zeros(0))
    bt = make_batch(g, net, n_tune, n_tune // 32, n_tune // 64, beta, nu, rho, s=s.copy())
    return net, bx, bt


def workload_paper_d1(M: int = 4000, n_tune: int = 65536, beta: float = 7.0):
    """The paper's convection setting in shape: LRNR of width M = 4,000 with ranks
    r = (1, 5, 5, 3, 1) (four hidden layers), pure convection with beta = 7; the fast
    phase samples X = the 4 x 3 cell-centred grid (12 interior points) and the
    fine-tune phase the collocation batch (n_tune interior, n_tune/32 initial,
    n_tune/64 periodic pairs).  Returns (net, batch_X, batch_tune)."""
    return _paper_workload(1005, M, [1, 5, 5, 3, 1], (beta, 0.0, 0.0), n_tune)


def workload_paper_d2(M: int = 4000, n_tune: int = 65536, mu=(2.0, 1.0, 1.0)):
    """The paper's convection-diffusion-reaction setting in shape: width M = 4,000,
    ranks r = (1, 49, 30, 25, 1), mu = (2, 1, 1) inside its parameter box
    [(1, 0, 0), (3, 2, 2)]; sample sets as in ``workload_paper_d1``."""
    return _paper_workload(1006, M, [1, 49, 30, 25, 1], mu, n_tune)


def snapshot_design(g: np.random.Generator, n_per_point: int = 8, std: float = 0.05):
    """EIM sample design: a 4 (x) x 3 (t) cell-centred grid plus Gaussian perturbations.

    Returns (x, t) of the 12 grid points followed by ``n_per_point`` perturbed copies
    of each, clipped into the closed domain.
    """
    gx = TWO_PI * (np.arange(4) + 0.5) / 4.0
    gt = (np.arange(3) + 0.5) / 3.0
    X, T = np.meshgrid(gx, gt, indexing="ij")
    x0, t0 = X.ravel(), T.ravel()
    xs, ts = [x0], [t0]
    for _ in range(n_per_point):
        xs.append(np.clip(x0 + g.normal(0.0, std * TWO_PI, size=x0.shape), 0.0, TWO_PI))
        ts.append(np.clip(t0 + g.normal(0.0, std, size=t0.shape), 0.0, 1.0))
    return np.concatenate(xs), np.concatenate(ts)
