"""Exact solvers for the replica Ising lattice: the oracle's own pins.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* ``replica_links``      -- the link set of the replica lattice of section 3
                            (eq. for H/T with couplings beta^(k,k), beta^(k,k+1)).
* ``log_z_enumerate``    -- ln Z by brute-force enumeration of all states.
* ``log_z2_transfer``    -- ln Z_2(l) by a transfer matrix along Euclidean time.
* ``log_z_kaufman``      -- ln Z of the periodic 2D Ising torus in closed form
                            (Kaufman 1949, ref. cited in section 4).
* ``exact_path_measure`` -- the exact distribution of (final state, W_int) of the
                            non-equilibrium Metropolis dynamics of Appendix A,
                            propagated state by state for tiny lattices.

Sites are numbered in the natural order ((r * L_t + t) * L_y + y) * L + x with
n = 2 replicas; the cut is at tau_c = 0 (links t = 0 -> 1), region A = {x < l},
and the switched column is x = l (section 3, protocol paragraph).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy import sparse

N_REPLICA = 2


def _site(L, L_t, L_y, r, t, y, x):
    return ((r * L_t + t) * L_y + y) * L + x


@dataclass
class Links:
    """Links of the replica lattice, each an (i, j) site pair.

    full: couplings fixed at beta; self_: the switched column's links inside a
    replica, coupling beta (1 - lambda); glue: the switched column's links to the
    next replica, coupling beta lambda (section 3, linear protocol)."""
    full: np.ndarray
    self_: np.ndarray
    glue: np.ndarray
    n_sites: int


def replica_links(d: int, L: int, L_t: int, l: int, n: int = N_REPLICA,
                  whole: bool = False) -> Links:
    """Every link once, from each site towards +x, +y (3D) and +t, for n
    replicas.

    The +t link leaving t = 0 crosses the cut: for x < l it lands in replica
    r + 1 (mod n, glued), for x > l in replica r, and for x = l both links
    exist with the switched couplings (section 3, replica H/T and the linear
    protocol).  whole: Alba et al.'s whole-cut transformation (section 3), the
    columns x < l switch and nothing is glued beforehand.
    """
    L_y = L if d == 3 else 1
    g0, g1 = (0, l) if whole else (l, l + 1)
    full, self_, glue = [], [], []
    for r in range(n):
        for t in range(L_t):
            for y in range(L_y):
                for x in range(L):
                    i = _site(L, L_t, L_y, r, t, y, x)
                    full.append((i, _site(L, L_t, L_y, r, t, y, (x + 1) % L)))
                    if d == 3:
                        full.append((i, _site(L, L_t, L_y, r, t, (y + 1) % L_y, x)))
                    tn = (t + 1) % L_t
                    same = _site(L, L_t, L_y, r, tn, y, x)
                    if t != 0:
                        full.append((i, same))
                        continue
                    other = _site(L, L_t, L_y, (r + 1) % n, tn, y, x)
                    if x < g0:
                        full.append((i, other))
                    elif x >= g1:
                        full.append((i, same))
                    else:
                        self_.append((i, same))
                        glue.append((i, other))
    as_arr = lambda v: np.array(v, dtype=np.int64).reshape(-1, 2)
    return Links(as_arr(full), as_arr(self_), as_arr(glue), n * L_t * L_y * L)


def _spins_of_states(n_sites: int) -> np.ndarray:
    """sigma[state, i] = +1 if bit i of state is 0 else -1 (int8)."""
    states = np.arange(1 << n_sites, dtype=np.int64)
    bits = (states[:, None] >> np.arange(n_sites, dtype=np.int64)[None, :]) & 1
    return (1 - 2 * bits).astype(np.int8)


def _bond_sums(sigma: np.ndarray, pairs: np.ndarray) -> np.ndarray:
    if len(pairs) == 0:
        return np.zeros(sigma.shape[0], dtype=np.int64)
    return (sigma[:, pairs[:, 0]].astype(np.int64) * sigma[:, pairs[:, 1]]).sum(axis=1)


def _logsumexp(v: np.ndarray) -> float:
    m = float(np.max(v))
    return m + math.log(float(np.sum(np.exp(v - m))))


def log_z_enumerate(d: int, L: int, L_t: int, l: int, beta: float, lam: float = 0.0,
                    n: int = N_REPLICA, whole: bool = False) -> float:
    """ln Z_n of the replica lattice at protocol parameter lambda by summing
    exp(-H/T) over all 2^V states (H/T of section 3 with the switched
    columns' couplings beta (1 - lambda), beta lambda).  V <= 20."""
    lk = replica_links(d, L, L_t, l, n, whole)
    sigma = _spins_of_states(lk.n_sites)
    e = (_bond_sums(sigma, lk.full) + (1.0 - lam) * _bond_sums(sigma, lk.self_)
         + lam * _bond_sums(sigma, lk.glue))
    return _logsumexp(beta * e)


def log_z_single_enumerate(d: int, L: int, L_t: int, beta: float) -> float:
    """ln Z of one periodic L^(d-1) x L_t Ising lattice by enumeration (eq. Ising_model)."""
    L_y = L if d == 3 else 1
    n = L_t * L_y * L
    sigma = _spins_of_states(n)
    pairs = []
    for t in range(L_t):
        for y in range(L_y):
            for x in range(L):
                i = (t * L_y + y) * L + x
                pairs.append((i, (t * L_y + y) * L + (x + 1) % L))
                if d == 3:
                    pairs.append((i, (t * L_y + (y + 1) % L_y) * L + x))
                pairs.append((i, (((t + 1) % L_t) * L_y + y) * L + x))
    return _logsumexp(beta * _bond_sums(sigma, np.array(pairs)))


# ----------------------------------------------------------- transfer matrix --
def _slice_transfer(d: int, L: int, beta: float):
    """Transfer matrix T(a, b) = w_space(a) w_time(a, b) between consecutive time
    slices of one replica, normalised by its largest eigenvalue (ratios of
    partition functions at equal L_t are unaffected).  Returns (T, column_of_bit)."""
    L_y = L if d == 3 else 1
    S = L * L_y
    sig = _spins_of_states(S).astype(np.int64)        # bit (y * L + x)
    space = np.zeros(1 << S, dtype=np.int64)
    for y in range(L_y):
        for x in range(L):
            i = y * L + x
            space += sig[:, i] * sig[:, y * L + (x + 1) % L]
            if d == 3:
                space += sig[:, i] * sig[:, ((y + 1) % L_y) * L + x]
    overlap = sig @ sig.T                               # sum_x a(x) b(x)
    T = np.exp(beta * space)[:, None] * np.exp(beta * overlap)
    lam_max = np.max(np.abs(np.linalg.eigvals(T)))
    column = np.array([i % L for i in range(S)])
    return T / lam_max, column


def log_z2_transfer(d: int, L: int, L_t: int, ls, beta: float) -> np.ndarray:
    """ln Z_2(l) (up to an l-independent constant) for each l in ls.

    Away from the cut both replicas evolve with T^(L_t) from slice t = 1 around
    to the cut; the cut swaps the columns x < l of the two replicas' t = 1
    slices (section 3: glue links join replica r at t = 0 to replica r+1 at
    t = 1).  Hence Z_2(l) = sum_{a,b} P(a, mix(b, a)) P(b, mix(a, b)) with
    P = T^(L_t) and mix(u, v) = u on columns x < l, v elsewhere.  The constant
    is the same for every l at fixed (d, L, L_t, beta), so differences are exact.
    """
    T, column = _slice_transfer(d, L, beta)
    P = np.linalg.matrix_power(T, L_t)
    n = P.shape[0]
    a = np.arange(n, dtype=np.int64)
    out = []
    for l in ls:
        mask = 0
        for bit, col in enumerate(column):
            if col < l:
                mask |= 1 << bit
        A, B = np.meshgrid(a, a, indexing="ij")
        mix_ba = (B & mask) | (A & ~mask)
        mix_ab = (A & mask) | (B & ~mask)
        z = np.sum(P[A, mix_ba] * P[B, mix_ab])
        out.append(math.log(z))
    return np.array(out)


def log_zn_transfer(d: int, L: int, L_t: int, ls, beta: float, n: int) -> np.ndarray:
    """ln Z_n(l) for n replicas (up to an l-independent constant), l in ls.

    Generalises log_z2_transfer: with P = T^(L_t) and M_l(u, v) = P(v, mix(u, v))
    (v's propagation closes on the slice that takes the previous replica's
    columns x < l), the replicas form a ring, so Z_n(l) = Tr M_l^n; for n = 2
    this is log_z2_transfer's double sum, and for l = 0 it is (Tr P)^n = Z^n.
    """
    T, column = _slice_transfer(d, L, beta)
    P = np.linalg.matrix_power(T, L_t)
    m = P.shape[0]
    a = np.arange(m, dtype=np.int64)
    U, V = np.meshgrid(a, a, indexing="ij")
    out = []
    for l in ls:
        mask = 0
        for bit, col in enumerate(column):
            if col < l:
                mask |= 1 << bit
        M = P[V, (U & mask) | (V & ~mask)]
        out.append(math.log(np.trace(np.linalg.matrix_power(M, n))))
    return np.array(out)


def delta_sn_transfer(d: int, L: int, L_t: int, beta: float, n: int) -> np.ndarray:
    """Exact Delta S_n(l -> l+1) = -ln[Z_n(l+1)/Z_n(l)]/(n-1), l = 0..L-1
    (section 2, eq. definition_of_derivative_of_Renyi_entropy with epsilon = a)."""
    lz = log_zn_transfer(d, L, L_t, range(L + 1), beta, n)
    return -(lz[1:] - lz[:-1]) / (n - 1)


def renyi_sn_transfer(d: int, L: int, L_t: int, beta: float, n: int) -> np.ndarray:
    """Exact S_n(l) = ln[Z_n(l)/Z^n]/(1-n) for l = 0..L (section 2, eq.
    trace_of_rho_n_as_ratio_of_partition_functions); S_n(0) = 0."""
    lz = log_zn_transfer(d, L, L_t, range(L + 1), beta, n)
    return (lz - lz[0]) / (1 - n)


def delta_s2_transfer(d: int, L: int, L_t: int, beta: float) -> np.ndarray:
    """Exact Delta S_2(l -> l+1) = -ln[Z_2(l+1)/Z_2(l)] for l = 0..L-1
    (section 2, eq. trace_of_rho_n_as_ratio_of_partition_functions with n = 2)."""
    lz = log_z2_transfer(d, L, L_t, range(L + 1), beta)
    return -(lz[1:] - lz[:-1])


# ----------------------------------------------------------------- Kaufman ---
def log_z_kaufman(m: int, n: int, beta: float) -> float:
    """ln Z of the periodic m x n square-lattice Ising model, coupling K = beta,
    from Kaufman's solution (Phys. Rev. 76 (1949) 1232; the paper's ref. for
    the 2D model in section 4):

        Z = 1/2 (2 sinh 2K)^(mn/2) [Z1 + Z2 + Z3 + Z4],
        Z1 = prod_{r<n} 2 cosh(m g_{2r+1}/2),  Z2 = prod 2 sinh(m g_{2r+1}/2),
        Z3 = prod_{r<n} 2 cosh(m g_{2r}/2),    Z4 = prod 2 sinh(m g_{2r}/2),
        cosh g_k = cosh 2K coth 2K - cos(pi k / n)  (k > 0),
        g_0 = 2K + ln tanh K  (signed).
    """
    K = beta
    c = math.cosh(2 * K) / math.tanh(2 * K)

    def gamma(k):
        if k == 0:
            return 2 * K + math.log(math.tanh(K))
        return math.acosh(c - math.cos(math.pi * k / n))

    logs = []
    signs = []
    for parity, fn in ((1, "cosh"), (1, "sinh"), (0, "cosh"), (0, "sinh")):
        lg, sg = 0.0, 1.0
        for r in range(n):
            g = gamma(2 * r + parity)
            v = 2 * (math.cosh(m * g / 2) if fn == "cosh" else math.sinh(m * g / 2))
            if v == 0.0:
                lg, sg = -math.inf, 0.0
                break
            lg += math.log(abs(v))
            sg *= math.copysign(1.0, v)
        logs.append(lg)
        signs.append(sg)
    top = max(lg for lg in logs if lg > -math.inf)
    total = sum(s * math.exp(lg - top) for s, lg in zip(signs, logs) if lg > -math.inf)
    return math.log(0.5) + (m * n / 2) * math.log(2 * math.sinh(2 * K)) + top + math.log(total)


# ------------------------------------------------------ exact path measure ---
def _threshold(beta: float, m: int, n_step: int | None) -> int:
    """The 32-bit Metropolis threshold floor(2^32 exp(-x)) saturated at 2^32 - 1,
    x = 2 beta m (bulk) or (2 beta m)/N (switched site); flips with probability
    T / 2^32."""
    if n_step is None:
        x = 2.0 * beta * float(m)
    else:
        x = (2.0 * beta * float(m)) / float(n_step)
    return min(int(math.floor(math.ldexp(math.exp(-x), 32))), 2 ** 32 - 1)


class _Schedule:
    """Which couplings of the switched columns (x = l, y) move at protocol
    step k.  Protocol 1 (section 3): every column together, lambda_{k+1} =
    (k+1)/N.  Protocol 2 (Appendix B): column y alone during the m = N/L_y
    steps y m .. (y+1) m - 1, with lambda = (k + 1 - y m)/m; columns already
    switched sit at the end geometry, the others at the start geometry."""

    def __init__(self, d, L, n_step, direction, protocol):
        self.L, self.L_y = L, (L if d == 3 else 1)
        self.dir, self.protocol = direction, protocol
        if protocol == 2 and n_step % self.L_y:
            raise ValueError("protocol 2 needs n_step to be a multiple of L_y")
        self.m = n_step // self.L_y if protocol == 2 else n_step

    def site_y(self, i: int) -> int:
        return (int(i) // self.L) % self.L_y

    def column(self, y: int, k) -> str:
        """'self', 'glue' or 'switching' for column y at step k (None: the
        start geometry, lambda = 0 forward, 1 reverse)."""
        if k is None:
            return "self" if self.dir > 0 else "glue"
        if self.protocol != 2:
            return "switching"
        active = k // self.m
        if y == active:
            return "switching"
        return "glue" if (y < active) == (self.dir > 0) else "self"

    def weights(self, k: int):
        """(den, w_self, w_glue): the switching column's couplings at step k
        are beta w_self/den and beta w_glue/den (lambda_{k+1})."""
        kp = k + 1 - (k // self.m) * self.m
        den = self.m
        return (den, den - kp, kp) if self.dir > 0 else (den, kp, den - kp)

    def work_rows(self, k: int, n_links: int, lower_sites) -> tuple:
        """Mask of the switched links whose couplings move at step k and the
        factor that puts their work in units of beta/N."""
        if self.protocol != 2:
            return np.ones(n_links, dtype=bool), 1
        active = k // self.m
        ys = np.array([self.site_y(i) for i in lower_sites], dtype=np.int64)
        return ys == active, self.L_y


class _Dynamics:
    """Single-site Metropolis probabilities of every site in every state of a
    tiny replica lattice, at the start geometry or at protocol step k."""

    def __init__(self, d, L, L_t, l, beta, n_step, direction, quantised, protocol=1,
                 n=N_REPLICA, whole=False):
        self.d, self.L, self.L_t, self.l = d, L, L_t, l
        self.beta, self.N, self.dir = beta, n_step, direction
        self.quantised = quantised
        self.sched = _Schedule(d, L, n_step, direction, protocol)
        self._cache = {}
        self.links = replica_links(d, L, L_t, l, n, whole)
        self.V = self.links.n_sites
        self.sigma = _spins_of_states(self.V).astype(np.int64)
        L_y = L if d == 3 else 1
        self.colour = np.zeros(self.V, dtype=np.int64)
        for r in range(n):
            for t in range(L_t):
                for y in range(L_y):
                    for x in range(L):
                        self.colour[_site(L, L_t, L_y, r, t, y, x)] = (x + y + t) % 2
        # per-site neighbour lists by link class (links are undirected)
        self.nb = {cls: [[] for _ in range(self.V)] for cls in ("full", "self", "glue")}
        for cls, pairs in (("full", self.links.full), ("self", self.links.self_),
                           ("glue", self.links.glue)):
            for i, j in pairs:
                self.nb[cls][i].append(j)
                self.nb[cls][j].append(i)

    def flip_prob(self, i: int, k: int | None) -> np.ndarray:
        """P(flip site i | state) for all states.  k = None: thermalisation at
        the start geometry (forward: self-linked column, reverse: glued)."""
        key = (i, k)
        if key not in self._cache:
            self._cache[key] = self._flip_prob(i, k)
        return self._cache[key]

    def _flip_prob(self, i: int, k: int | None) -> np.ndarray:
        s = self.sigma
        a = np.zeros(s.shape[0], dtype=np.int64)
        for j in self.nb["full"][i]:
            a += s[:, i] * s[:, j]
        special = bool(self.nb["self"][i])
        col = self.sched.column(self.sched.site_y(i), k) if special else None
        if special and col != "switching":
            # a column at the start or end geometry is a bulk site
            for j in self.nb[col][i]:
                a += s[:, i] * s[:, j]
            special = False
        if not special:
            m = a
            x = 2.0 * self.beta * m
            nstep = None
        else:
            (js,), (jg,) = self.nb["self"][i], self.nb["glue"][i]
            b = s[:, i] * s[:, js]
            c = s[:, i] * s[:, jg]
            den, w_self, w_glue = self.sched.weights(k)   # step k updates at lambda_{k+1}
            m = a * den + b * w_self + c * w_glue
            x = (2.0 * self.beta * m) / den
            nstep = den
        if self.quantised:
            um, inv = np.unique(m, return_inverse=True)
            pu = np.array([1.0 if mm <= 0 else _threshold(self.beta, int(mm), nstep) / 2.0 ** 32
                           for mm in um])
            p = pu[inv.reshape(-1)]
        else:
            p = np.minimum(1.0, np.exp(-x))
        return p

    def sweep(self, f: np.ndarray, k: int | None) -> np.ndarray:
        """Apply one checkerboard sweep (colour 0 then colour 1) to a density f
        over states (last axis).  Sites of one colour are independent given the
        other colour, so their single-site kernels are applied one after another."""
        for col in (0, 1):
            for i in np.nonzero(self.colour == col)[0]:
                p = self.flip_prob(int(i), k)
                partner = np.arange(f.shape[-1]) ^ (1 << int(i))
                f = f * (1.0 - p) + (f * p)[..., partner]
        return f

    def work_increment(self, k: int = 0) -> np.ndarray:
        """dE(state) with dW_k = (beta/N) dE = H_{k+1} - H_k (Appendix A, eq.
        work_in_one_MC_step): sum over the switched links that move at step k
        of (self - glue) bond products, in units of beta/N, sign flipped for
        the reverse protocol."""
        return _work_increment(self.sigma, self.links, self.sched, k)

    def energy(self, lam: float) -> np.ndarray:
        lk = self.links
        return -(_bond_sums(self.sigma, lk.full) + (1 - lam) * _bond_sums(self.sigma, lk.self_)
                 + lam * _bond_sums(self.sigma, lk.glue))


def _work_increment(sigma, links, sched, k):
    sel, factor = sched.work_rows(k, len(links.self_), links.self_[:, 0])
    e = factor * (_bond_sums(sigma, links.self_[sel]) - _bond_sums(sigma, links.glue[sel]))
    return e if sched.dir > 0 else -e


def _propagate(F, de):
    """Shift the work axis of F by dE(state) (W index = W_int + offset)."""
    G = np.zeros_like(F)
    for dv in np.unique(de):
        sel = de == dv
        if dv >= 0:
            G[dv:, sel] += F[:F.shape[0] - dv, sel]
        else:
            G[:dv, sel] += F[-dv:, sel]
    return G


def exact_path_measure(d, L, L_t, l, beta, n_step, n_sweep, n_therm, *, direction=1,
                       quantised=True, start="hot", protocol=1, n=N_REPLICA, whole=False,
                       therm="metropolis"):
    """Exact joint law of (W_int, final state) of the non-equilibrium dynamics.

    start="hot": uniform start (independent random spins) followed by n_therm
    sweeps at the start geometry, as the Monte Carlo trajectories do --
    Metropolis sweeps, or with therm="sw" exact Swendsen-Wang steps (Appendix A
    asks only for an equilibrium start; section 4 thermalises with cluster
    steps); start="equilibrium": exact Boltzmann weights pi_{lambda_0}
    (Appendix A, eq. equilibrium_distribution), for the Jarzynski identity.
    The protocol sweeps are Metropolis sweeps.
    Returns (w_values, F) with F[w_index, state] the probability.
    """
    dyn = _Dynamics(d, L, L_t, l, beta, n_step, direction, quantised, protocol, n, whole)
    n_states = 1 << dyn.V
    lam0 = 0.0 if direction > 0 else 1.0
    if start == "hot" and therm == "sw":
        f = np.full(n_states, 1.0 / n_states)
        T0 = _SWDynamics(d, L, L_t, l, beta, n_step, direction, quantised, protocol, n,
                         whole).kernel(None)
        for _ in range(n_therm):
            f = f @ T0
    elif start == "hot":
        f = np.full(n_states, 1.0 / n_states)
        for _ in range(n_therm):
            f = dyn.sweep(f, None)
    else:
        e = -beta * dyn.energy(lam0)
        w = np.exp(e - e.max())
        f = w / w.sum()
    des = [dyn.work_increment(k) for k in range(n_step)]
    wmax = sum(int(np.max(np.abs(de))) for de in des)
    F = np.zeros((2 * wmax + 1, n_states))
    F[wmax] = f
    for k in range(n_step):
        F = _propagate(F, des[k])
        for _ in range(n_sweep):
            F = dyn.sweep(F, k)
    return np.arange(-wmax, wmax + 1), F


# ----------------------------------------------- exact Swendsen-Wang kernel --
def _bond_prob(x: float, quantised: bool) -> float:
    """Swendsen-Wang bond probability 1 - e^{-x} (x = 2K) between equal spins;
    quantised: floor(2^32 (1 - e^{-x})) / 2^32, saturated at 1 - 2^-32."""
    if quantised:
        return min(int(math.floor(math.ldexp(-math.expm1(-x), 32))), 2 ** 32 - 1) / 2.0 ** 32
    return -math.expm1(-x)


class _SWDynamics:
    """Exact Swendsen-Wang transition matrices of a tiny replica lattice
    (Swendsen and Wang 1987, the update of the paper's GPU code, section 3):
    every link of coupling K between equal spins is a bond with probability
    1 - e^{-2K}; each cluster of bonded sites flips with probability 1/2.
    T[s, s'] = sum over bond sets B of P(B | s) 2^{-nc(B)} [s' = s with some
    clusters of B flipped], computed by enumerating all bond sets."""

    def __init__(self, d, L, L_t, l, beta, n_step, direction, quantised, protocol=1,
                 n=N_REPLICA, whole=False):
        self.beta, self.N, self.dir, self.quantised = beta, n_step, direction, quantised
        self.sched = _Schedule(d, L, n_step, direction, protocol)
        self.links = replica_links(d, L, L_t, l, n, whole)
        self.V = self.links.n_sites
        if self.V > 10:
            raise ValueError("exact Swendsen-Wang kernel needs V <= 10")
        lk = self.links
        self.pairs = np.concatenate([lk.full, lk.self_, lk.glue])
        self.kind = np.array([0] * len(lk.full) + [1] * len(lk.self_) + [2] * len(lk.glue))
        self.link_y = np.array([self.sched.site_y(i) for i in self.pairs[:, 0]])
        self.sigma = _spins_of_states(self.V).astype(np.int64)
        self.aligned = (self.sigma[:, self.pairs[:, 0]] == self.sigma[:, self.pairs[:, 1]])
        self._cache = {}

    def _x(self, kind, k, y):
        """x = 2K of a link of class kind in column y at protocol step k (None:
        thermalisation at the start geometry)."""
        b = self.beta
        if kind == 0:
            return 2.0 * b
        col = self.sched.column(y, k)
        if col != "switching":
            return 2.0 * b if col == ("self" if kind == 1 else "glue") else 0.0
        den, w_self, w_glue = self.sched.weights(k)
        w = w_self if kind == 1 else w_glue
        return (2.0 * b * float(w)) / float(den)

    def kernel(self, k):
        if k in self._cache:
            return self._cache[k]
        p = np.array([_bond_prob(self._x(kd, k, y), self.quantised)
                      for kd, y in zip(self.kind, self.link_y)])
        live = np.nonzero(p > 0)[0]
        pairs, pl = self.pairs[live], p[live]
        nl, n_states, V = len(live), 1 << self.V, self.V
        aligned = self.aligned[:, live]
        # every bond set B of the live links: membership and cluster labels
        # (label = smallest site index of the component, by V rounds of min
        # propagation along the bonds of B)
        subsets = np.arange(1 << nl, dtype=np.int64)
        inB = ((subsets[:, None] >> np.arange(nl)[None, :]) & 1).astype(bool)
        lab = np.tile(np.arange(V), (1 << nl, 1))
        for _ in range(V):
            for e in range(nl):
                i, j = pairs[e]
                m = np.minimum(lab[:, i], lab[:, j])
                sel = inB[:, e]
                lab[sel, i] = m[sel]
                lab[sel, j] = m[sel]
        parts, pid = np.unique(lab, axis=0, return_inverse=True)
        pid = pid.reshape(-1)
        # P(B | s) = prod_{e in B} [aligned_e(s)] p_e * prod_{e not in B} (1 - [aligned_e(s)] p_e);
        # W[partition, s] = sum of P(B | s) over the bond sets B with that partition
        log_p = np.log(pl)
        log_q = np.log1p(-(aligned * pl[None, :])).T                    # (links, states)
        unequal = (~aligned).astype(np.float64).T                         # (links, states)
        W = np.zeros((len(parts), n_states))
        chunk = 16384
        for lo in range(0, 1 << nl, chunk):
            b = inB[lo:lo + chunk].astype(np.float64)
            prob = np.exp((b @ log_p)[:, None] + (1.0 - b) @ log_q)
            prob[(b @ unequal) > 0] = 0.0                                 # a bond between unequal spins
            ind = sparse.csr_matrix((np.ones(len(b)), (pid[lo:lo + chunk], np.arange(len(b)))),
                                    shape=(len(parts), len(b)))
            W += ind @ prob
        T = np.zeros((n_states, n_states))
        s_idx = np.arange(n_states)
        for q, row in enumerate(parts):
            roots = np.unique(row)
            masks = np.array([sum(1 << i for i in range(V) if row[i] == r) for r in roots])
            nc = len(masks)
            sel = (np.arange(1 << nc)[:, None] >> np.arange(nc)[None, :]) & 1
            flips = np.bitwise_or.reduce(sel * masks[None, :], axis=1)
            T[s_idx[:, None], s_idx[:, None] ^ flips[None, :]] += W[q][:, None] / (1 << nc)
        self._cache[k] = T
        return T

    def work_increment(self, k: int = 0):
        return _work_increment(self.sigma, self.links, self.sched, k)

    def energy(self, lam):
        lk = self.links
        return -(_bond_sums(self.sigma, lk.full) + (1 - lam) * _bond_sums(self.sigma, lk.self_)
                 + lam * _bond_sums(self.sigma, lk.glue))


def exact_path_measure_sw(d, L, L_t, l, beta, n_step, n_sweep, n_therm, *, direction=1,
                          quantised=True, start="hot", protocol=1, n=N_REPLICA, whole=False):
    """Exact joint law of (W_int, final state) of the non-equilibrium dynamics
    with Swendsen-Wang updates (same protocol as exact_path_measure: work
    before each update, update at lambda_{k+1}).  Returns (w_values, F)."""
    dyn = _SWDynamics(d, L, L_t, l, beta, n_step, direction, quantised, protocol, n, whole)
    n_states = 1 << dyn.V
    lam0 = 0.0 if direction > 0 else 1.0
    if start == "hot":
        f = np.full(n_states, 1.0 / n_states)
        T0 = dyn.kernel(None)
        for _ in range(n_therm):
            f = f @ T0
    else:
        e = -beta * dyn.energy(lam0)
        w = np.exp(e - e.max())
        f = w / w.sum()
    des = [dyn.work_increment(k) for k in range(n_step)]
    wmax = sum(int(np.max(np.abs(de))) for de in des)
    F = np.zeros((2 * wmax + 1, n_states))
    F[wmax] = f
    for k in range(n_step):
        F = _propagate(F, des[k])
        Tk = dyn.kernel(k)
        for _ in range(n_sweep):
            F = F @ Tk
    return np.arange(-wmax, wmax + 1), F
