"""Independent restatements of the sorption-MP method as explicit Markov chains.

A tracer of the method performs a Markov chain on the states {free at a fluid node r} and
{adsorbed at an interfacial node r}. From a free state it jumps along link i with
probability p_i(r) (only to fluid nodes), adsorbs with p_a at interfacial nodes, else stays;
an adsorbed tracer desorbs in place with p_d. Every propagated quantity of the paper is a
vector over these states multiplied by powers of the chain's transition matrix, and the
VACF is <v(0) v(t)> over chain paths started from the Boltzmann weights.

These builders are written from that description, not from the stencil form the oracle
uses, so agreement between the two pins the oracle's indexing, signs and terms:
  * dense_chain   -- the full chain of a small 3D lattice (dense matrix, any geometry/flow);
  * z_chain       -- a slit (x,y-invariant) reduced exactly to its H+2 z-states;
  * walkers       -- seeded random walkers sampling the dense chain.
Their own D3Q19 table is checked against the lattice identities in the tests.
"""
from __future__ import annotations

import itertools

import numpy as np

# D3Q19 moving links written out as all c in {-1,0,1}^3 with |c|^2 in {1, 2}
C18 = np.array([c for c in itertools.product((-1, 0, 1), repeat=3)
                if 1 <= sum(abs(v) for v in c) <= 2], dtype=np.int64)
W18 = np.where((np.abs(C18).sum(1)) == 1, 1.0 / 18.0, 1.0 / 36.0)


def move_prob(u, lam):
    """Probability of each of the 18 moves from a node with velocity u (before closing
    links into solids): w (lam/2) + w (3 c.u + 9/2 (c.u)^2 - 3/2 u.u)."""
    cu = C18 @ np.asarray(u, dtype=np.float64)
    uu = float(np.dot(u, u))
    return W18 * (lam / 2.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu)


class Chain:
    """Transition list of a finite chain: T[a, b] and per-transition increments."""

    def __init__(self, nstates):
        self.n = nstates
        self.T = np.zeros((nstates, nstates))
        self.inc = np.zeros((3, nstates, nstates))  # displacement of a->b (well defined here)
        self.rows = [[] for _ in range(nstates)]    # (b, prob, (dx,dy,dz)) for walkers

    def add(self, a, b, p, d):
        self.T[a, b] += p
        self.inc[:, a, b] = d
        self.rows[a].append((b, p, tuple(d)))

    def vacf(self, pi0, g, tmax):
        """Z_g(t), t = 0..tmax, for a chain started from the distribution pi0 with the
        velocity of step t the increment of the jump t -> t+1."""
        V = self.T * self.inc[g]
        m = V.sum(1)                      # mean increment from each state
        Z = np.zeros(tmax + 1)
        Z[0] = pi0 @ (self.T * self.inc[g] ** 2).sum(1)
        w = pi0 @ V                       # v(0)-weighted occupation after one step
        for t in range(1, tmax + 1):
            Z[t] = w @ m
            w = w @ self.T
        return Z

    def asymptotic_K(self, pi0, g):
        """K = (Z0 - Zinf)/2 + sum_{m>=1} (Z_m - Zinf), Zinf = vbar^2, with pi0 stationary,
        from one linear solve of the chain's Poisson equation (I - T) h = m - vbar."""
        V = self.T * self.inc[g]
        m = V.sum(1)
        vbar = pi0 @ m
        Z0 = pi0 @ (self.T * self.inc[g] ** 2).sum(1)
        A = np.vstack([np.eye(self.n) - self.T, pi0[None, :]])
        rhs = np.concatenate([m - vbar, [0.0]])
        h, *_ = np.linalg.lstsq(A, rhs, rcond=None)
        w = pi0 @ V
        return (Z0 - vbar ** 2) / 2.0 + w @ h, vbar


def dense_chain(solid, u, D_b, k_a, k_d):
    """Full chain of a small periodic lattice. solid[nz,ny,nx]; u[3,nz,ny,nx] or None.
    Returns (chain, free_index[N] (-1 on solid), ads_index[N] (-1 off the interface),
    pi0 over states from the Boltzmann weights)."""
    nz, ny, nx = solid.shape
    lam = 12.0 * D_b
    fluid = ~solid.astype(bool)
    coords = [(z, y, x) for z in range(nz) for y in range(ny) for x in range(nx)]
    free = -np.ones(solid.size, dtype=np.int64)
    ads = -np.ones(solid.size, dtype=np.int64)
    k = 0
    for n, (z, y, x) in enumerate(coords):
        if fluid[z, y, x]:
            free[n] = k
            k += 1

    def lin(z, y, x):
        return ((z % nz) * ny + (y % ny)) * nx + (x % nx)

    iface = np.zeros(solid.size, dtype=bool)
    for n, (z, y, x) in enumerate(coords):
        if fluid[z, y, x]:
            iface[n] = any(solid[(z + c[2]) % nz, (y + c[1]) % ny, (x + c[0]) % nx] for c in C18)
    for n in range(solid.size):
        if iface[n]:
            ads[n] = k
            k += 1
    ch = Chain(k)
    for n, (z, y, x) in enumerate(coords):
        if not fluid[z, y, x]:
            continue
        a = free[n]
        uu = np.zeros(3) if u is None else u[:, z, y, x]
        pm = move_prob(uu, lam)
        out = 0.0
        for c, p in zip(C18, pm):
            tgt = lin(z + c[2], y + c[1], x + c[0])
            if fluid.reshape(-1)[tgt]:
                ch.add(a, free[tgt], p, c)
                out += p
        if iface[n]:
            ch.add(a, ads[n], k_a, (0, 0, 0))
            out += k_a
            ch.add(ads[n], a, k_d, (0, 0, 0))
            ch.add(ads[n], ads[n], 1.0 - k_d, (0, 0, 0))
        ch.add(a, a, 1.0 - out, (0, 0, 0))
    K = 0.0 if k_a == 0 else k_a / k_d
    pi0 = np.zeros(k)
    pi0[free[free >= 0]] = 1.0
    pi0[ads[ads >= 0]] = K
    pi0 /= pi0.sum()
    return ch, free, ads, pi0


def z_chain(H, ux_of_z, D_b, k_a, k_d):
    """Exact reduction of a slit (solid planes z = 0, H+1; flow u = (ux(z), 0, 0)) to the
    z-states free_1..free_H, ads_1, ads_H. Returns (chain, pi0)."""
    lam = 12.0 * D_b
    ch = Chain(H + 2)
    ads = {1: H, H: H + 1}
    for z in range(1, H + 1):
        a = z - 1
        pm = move_prob((ux_of_z[z], 0.0, 0.0), lam)
        out = 0.0
        for c, p in zip(C18, pm):
            zt = z + c[2]
            if 1 <= zt <= H:
                # several (x, y) moves land on the same z-state: increments differ, so
                # accumulate the increment-weighted probability, not the increment
                ch.T[a, zt - 1] += p
                ch.rows[a].append((zt - 1, p, tuple(c)))
                out += p
        if z in ads:
            ch.T[a, ads[z]] += k_a
            ch.rows[a].append((ads[z], k_a, (0, 0, 0)))
            out += k_a
            ch.T[ads[z], a] += k_d
            ch.rows[ads[z]].append((a, k_d, (0, 0, 0)))
            ch.T[ads[z], ads[z]] += 1.0 - k_d
            ch.rows[ads[z]].append((ads[z], 1.0 - k_d, (0, 0, 0)))
        ch.T[a, a] += 1.0 - out
        ch.rows[a].append((a, 1.0 - out, (0, 0, 0)))
    # increment-weighted matrices (several links can join the same pair of z-states)
    ch.Vg = np.zeros((3, ch.n, ch.n))
    ch.V2g = np.zeros((3, ch.n, ch.n))
    for a, row in enumerate(ch.rows):
        for b, p, d in row:
            for g in range(3):
                ch.Vg[g, a, b] += p * d[g]
                ch.V2g[g, a, b] += p * d[g] * d[g]
    K = 0.0 if k_a == 0 else k_a / k_d
    pi0 = np.ones(H + 2)
    pi0[H] = pi0[H + 1] = K
    pi0 /= pi0.sum()
    return ch, pi0


def zchain_vacf(ch, pi0, g, tmax):
    """Z_g(t) of a z-chain (uses the increment-weighted matrices)."""
    V = ch.Vg[g]
    m = V.sum(1)
    Z = np.zeros(tmax + 1)
    Z[0] = pi0 @ ch.V2g[g].sum(1)
    w = pi0 @ V
    for t in range(1, tmax + 1):
        Z[t] = w @ m
        w = w @ ch.T
    return Z


def zchain_K(ch, pi0, g):
    """Asymptotic K of a z-chain from its Poisson equation (pi0 stationary)."""
    V = ch.Vg[g]
    m = V.sum(1)
    vbar = pi0 @ m
    Z0 = pi0 @ ch.V2g[g].sum(1)
    A = np.vstack([np.eye(ch.n) - ch.T, pi0[None, :]])
    rhs = np.concatenate([m - vbar, [0.0]])
    h, *_ = np.linalg.lstsq(A, rhs, rcond=None)
    return (Z0 - vbar ** 2) / 2.0 + (pi0 @ V) @ h, vbar


def walkers(ch, pi0, nwalk, tmax, seed):
    """Seeded random walkers on a chain started from pi0. Returns the per-step
    displacements, shape (tmax+1, 3, nwalk) (float32 to bound memory)."""
    rng = np.random.default_rng(seed)
    width = max(len(r) for r in ch.rows)
    cum = np.ones((ch.n, width))
    tgt = np.zeros((ch.n, width), dtype=np.int64)
    dis = np.zeros((ch.n, width, 3))
    for a, row in enumerate(ch.rows):
        ps = np.array([p for _, p, _ in row])
        assert np.all(ps >= 0.0), "walkers need non-negative probabilities"
        cum[a, :len(row)] = np.cumsum(ps)
        cum[a, len(row) - 1:] = np.inf   # the last entry absorbs the rounding of the sum
        tgt[a, :len(row)] = [b for b, _, _ in row]
        tgt[a, len(row):] = a
        dis[a, :len(row)] = [d for _, _, d in row]
    state = rng.choice(ch.n, size=nwalk, p=pi0)
    steps = np.zeros((tmax + 1, 3, nwalk), dtype=np.float32)
    for t in range(tmax + 1):
        r = rng.random(nwalk)
        k = (r[:, None] >= cum[state]).sum(1)
        steps[t] = dis[state, k].T
        state = tgt[state, k]
    return steps



def zchain_D(ch, pi0, g, ts, confined=False):
    """D_g(t) = Z(0)/2 + sum_{m=1}^t Z(m) of a z-chain at the integer times ts, summed in
    closed form over the eigenvalues mu_k of the transition matrix. With Z(m) =
    sum_k a_k mu_k^(m-1) (a_k from the eigen-expansion of the chain started from pi0):
        D(t) = Z(0)/2 + sum_k a_k (1 - mu_k^t)/(1 - mu_k)      (mu_k = 1 terms: a_k t).
    confined=True (a direction in which the tracer cannot leave, so D(inf) = 0) sums only
    the decaying tails, D(t) = -sum_{mu_k != 1} a_k mu_k^t/(1 - mu_k), which keeps full
    relative accuracy where D(t) has decayed by many orders. A chain reversible with respect
    to pi0 (u = 0) is diagonalised symmetrically."""
    V = ch.Vg[g]
    m = V.sum(1)
    Z0 = pi0 @ ch.V2g[g].sum(1)
    w = pi0 @ V
    live = pi0 > 0.0                      # states the start can reach (no adsorbed ones if k_a = 0)
    P = pi0[live, None] * ch.T[np.ix_(live, live)]
    if np.max(np.abs(P - P.T)) < 1e-15:
        # S = Pi^(1/2) T Pi^(-1/2) is symmetric: T = Pi^(-1/2) Q diag(mu) Q^T Pi^(1/2)
        r = np.sqrt(pi0[live])
        mu, Q = np.linalg.eigh(ch.T[np.ix_(live, live)] * r[:, None] / r[None, :])
        a = ((w[live] / r) @ Q) * (Q.T @ (r * m[live]))
    else:
        mu, R = np.linalg.eig(ch.T.T)     # columns: left eigenvectors of T
        a = np.linalg.solve(R, w) * (R.T @ m)
    mu = mu.astype(np.complex128)
    a = a.astype(np.complex128)
    one = np.abs(1.0 - mu) < 1e-12
    ts = np.asarray(ts, dtype=np.float64)
    out = np.empty(ts.shape)
    for j, t in enumerate(ts):
        if confined:
            tail = a[~one] * mu[~one] ** t / (1.0 - mu[~one])
            out[j] = -np.real(np.sum(tail))
        else:
            geo = np.where(one, t, (1.0 - mu ** t) / np.where(one, 1.0, 1.0 - mu))
            out[j] = Z0 / 2.0 + np.real(np.sum(a * geo))
    return out
