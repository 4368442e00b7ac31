"""The channel of the flow-past-a-fiber benchmark (Sec. 5.3): MAC operators with inflow and
traction-outflow boundaries.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Domain [0, Lx) x [0, Ly], periodic in x, Nx x Ny square cells of side h.  Unknowns (3 Nx Ny,
the same count and block order as the periodic grid):
  u_{i,j}  at (i h, (j + 1/2) h),  i < Nx, j < Ny             index  j Nx + i
  v_{i,j}  at ((i + 1/2) h, j h),  i < Nx, j < Ny             index  Nx Ny + j Nx + i
           (row j = 0 lies on the outflow boundary y = 0; the faces on y = Ly are prescribed)
  p_{i,j}  at cell centres                                     index  2 Nx Ny + j Nx + i

Boundary conditions (Sec. 5.3):
  top    y = Ly:  u = u_top, v = v_top(x)  (the prescribed inflow)
  bottom y = 0:   sigma n = t, n = (0, -1), sigma = -p I + mu (grad u + grad u^T); the paper's
                  backflow term (rho/2) min(u.n, 0) u enters through t, evaluated at the old
                  velocity like the convective term.

Discretisation (readings; the paper states the boundary conditions, not their stencils):
the interior rows are the periodic grid's (Sec. 2): rho/dt u - mu L u + G p on velocity faces
and -D u on cells.  Values outside the unknowns enter through ghost values:
  * above the top row of u:  u_{i,Ny} = 2 u_top - u_{i,Ny-1}   (the wall value is the mean)
  * the prescribed v_{i,Ny} = v_top(x_{i+1/2})
  * below the bottom row of u, from the tangential traction -mu (du/dy + dv/dx) = t_x at
    (i h, 0):  u_{i,-1} = u_{i,0} + (v_{i,0} - v_{i-1,0}) + h t_x / mu
  * below the outflow row of v, from continuity in the ghost cell (i, -1):
    v_{i,-1} = v_{i,0} + (u_{i+1,-1} - u_{i,-1})
  * the ghost pressure, from the normal traction p - 2 mu dv/dy = t_y at y = 0 with
    p(0) = (p_{i,0} + p_{i,-1}) / 2 and dv/dy(0) = (v_{i,1} - v_{i,-1}) / (2h):
    p_{i,-1} = 2 t_y + 2 mu (v_{i,1} - v_{i,-1}) / h - p_{i,0}
and the outflow faces v_{i,0} take the full-cell momentum row with these ghosts.  The
traction boundary fixes the pressure level, so the system has no null space.

The pins reproduce, exactly, three discrete solutions the scheme must keep: uniform inflow
passing straight through the outflow, a linear shear layer against the inflow wall, and a
hydrostatic pressure column under a body force.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class Channel:
    Nx: int
    Ny: int
    h: float
    rho: float
    mu: float
    dt: float

    @property
    def n(self) -> int:
        return 3 * self.Nx * self.Ny

    def iu(self, i, j):
        return j * self.Nx + i % self.Nx

    def iv(self, i, j):
        return self.Nx * self.Ny + j * self.Nx + i % self.Nx

    def ip(self, i, j):
        return 2 * self.Nx * self.Ny + j * self.Nx + i % self.Nx


class _Lin:
    """A linear combination of unknowns plus a constant (for ghost values)."""

    def __init__(self, terms=None, const=0.0):
        self.t = dict(terms or {})
        self.c = const

    def __add__(self, o):
        o = o if isinstance(o, _Lin) else _Lin(const=float(o))
        t = dict(self.t)
        for k, v in o.t.items():
            t[k] = t.get(k, 0.0) + v
        return _Lin(t, self.c + o.c)

    def __rmul__(self, a):
        return _Lin({k: a * v for k, v in self.t.items()}, a * self.c)

    def __sub__(self, o):
        return self + (-1.0) * (o if isinstance(o, _Lin) else _Lin(const=float(o)))

    def __radd__(self, a):
        return self + a

    def __rsub__(self, a):
        return _Lin(const=float(a)) - self


def operator(ch: Channel, u_top=0.0, v_top=None, t_x=None, t_y=None, structural=False):
    """K0 (3 Nx Ny square, the Stokes part of K_E on the channel) and the boundary vector g,
    such that the discrete equations read  K0 w = b + g  for a right-hand side b (body force
    and rho/dt u^n on the velocity rows, 0 on the cells).  v_top: (Nx,) inflow at the top
    faces; t_x: (Nx,) tangential traction at the points (i h, 0); t_y: (Nx,) normal traction
    at ((i + 1/2) h, 0).  structural=True: K0 holds a 1 at every unknown a row's stencil
    reaches through the ghost rules, including those whose weights cancel (the outflow v
    row's v_{i+-1,0})."""
    Nx, Ny, h, mu = ch.Nx, ch.Ny, ch.h, ch.mu
    v_top = np.zeros(Nx) if v_top is None else np.asarray(v_top, dtype=np.float64)
    t_x = np.zeros(Nx) if t_x is None else np.asarray(t_x, dtype=np.float64)
    t_y = np.zeros(Nx) if t_y is None else np.asarray(t_y, dtype=np.float64)
    U = lambda i, j: _Lin({ch.iu(i, j): 1.0})  # noqa: E731
    V = lambda i, j: _Lin({ch.iv(i, j): 1.0})  # noqa: E731
    P = lambda i, j: _Lin({ch.ip(i, j): 1.0})  # noqa: E731

    def u_at(i, j):
        if j == Ny:
            return 2.0 * u_top - U(i, Ny - 1)
        if j == -1:
            return U(i, 0) + (V(i, 0) - V(i - 1, 0)) + h * t_x[i % Nx] / mu
        return U(i, j)

    def v_at(i, j):
        if j == Ny:
            return _Lin(const=v_top[i % Nx])
        if j == -1:
            return V(i, 0) + (u_at(i + 1, -1) - u_at(i, -1))
        return V(i, j)

    def p_at(i, j):
        if j == -1:
            return 2.0 * t_y[i % Nx] + (2.0 * mu / h) * (v_at(i, 1) - v_at(i, -1)) - P(i, 0)
        return P(i, j)

    rows, cols, vals = [], [], []
    g = np.zeros(ch.n)

    def emit(r, expr):
        for c, a in expr.t.items():
            if a != 0.0 or structural:
                rows.append(r)
                cols.append(c)
                vals.append(1.0 if structural else a)
        g[r] -= expr.c  # constants move to the right-hand side

    a0, ih2, ih = ch.rho / ch.dt, 1.0 / (h * h), 1.0 / h
    for j in range(Ny):
        for i in range(Nx):
            lap = (u_at(i + 1, j) + u_at(i - 1, j) + u_at(i, j + 1) + u_at(i, j - 1) - 4.0 * U(i, j))
            emit(ch.iu(i, j), a0 * U(i, j) - (mu * ih2) * lap + ih * (P(i, j) - P(i - 1, j)))
            lap = (v_at(i + 1, j) + v_at(i - 1, j) + v_at(i, j + 1) + v_at(i, j - 1) - 4.0 * V(i, j))
            emit(ch.iv(i, j), a0 * V(i, j) - (mu * ih2) * lap + ih * (p_at(i, j) - p_at(i, j - 1)))
            div = (u_at(i + 1, j) - u_at(i, j)) + (v_at(i, j + 1) - v_at(i, j))
            emit(ch.ip(i, j), (-ih) * div)
    K = sp.csr_matrix((vals, (rows, cols)), shape=(ch.n, ch.n))
    K.sum_duplicates()
    if structural:
        K.data[:] = 1.0
    return K, g


def fields(ch: Channel, u_fn, v_fn, p_fn) -> np.ndarray:
    """The unknown vector sampled from point functions (u at u faces, v at v faces, p at
    centres)."""
    w = np.zeros(ch.n)
    for j in range(ch.Ny):
        for i in range(ch.Nx):
            w[ch.iu(i, j)] = u_fn(i * ch.h, (j + 0.5) * ch.h)
            w[ch.iv(i, j)] = v_fn((i + 0.5) * ch.h, j * ch.h)
            w[ch.ip(i, j)] = p_fn((i + 0.5) * ch.h, (j + 0.5) * ch.h)
    return w


# --------------------------------------------------------------------------- multigrid (Sec. 4)

def prolong(chc: Channel) -> sp.csr_matrix:
    """RT0 / bilinear prolongation from the channel chc to the one with twice its cells per
    direction, as on the periodic grid (Sec. 4), with two boundary readings: a fine v row on a
    coarse cell's midline next to the inflow wall takes half the coarse face below it (the
    prescribed faces carry no correction), and the pressure's bilinear stencil is clamped to
    the boundary cells in y (constant extrapolation of the correction)."""
    Nxc, Nyc = chc.Nx, chc.Ny
    chf = Channel(2 * Nxc, 2 * Nyc, chc.h / 2, chc.rho, chc.mu, chc.dt)
    rows, cols, vals = [], [], []
    for j in range(chf.Ny):
        for i in range(chf.Nx):
            r = chf.iu(i, j)
            if i % 2 == 0:
                rows.append(r); cols.append(chc.iu(i // 2, j // 2)); vals.append(1.0)
            else:
                for I in ((i - 1) // 2, (i + 1) // 2):
                    rows.append(r); cols.append(chc.iu(I, j // 2)); vals.append(0.5)
            r = chf.iv(i, j)
            if j % 2 == 0:
                rows.append(r); cols.append(chc.iv(i // 2, j // 2)); vals.append(1.0)
            else:
                for J in ((j - 1) // 2, (j + 1) // 2):
                    if J < Nyc:
                        rows.append(r); cols.append(chc.iv(i // 2, J)); vals.append(0.5)
            r = chf.ip(i, j)
            J0, sj = j // 2, (-1 if j % 2 == 0 else 1)
            I0, si = i // 2, (-1 if i % 2 == 0 else 1)
            for (dI, dJ, wt) in ((0, 0, 9 / 16), (si, 0, 3 / 16), (0, sj, 3 / 16), (si, sj, 1 / 16)):
                J = min(max(J0 + dJ, 0), Nyc - 1)
                rows.append(r); cols.append(chc.ip(I0 + dI, J)); vals.append(wt)
    P = sp.csr_matrix((vals, (rows, cols)), shape=(chf.n, chc.n))
    P.sum_duplicates()
    return P


def restrict(chc: Channel) -> sp.csr_matrix:
    """(1/4) P^T on the velocities, the four-cell average on the pressure (Sec. 4)."""
    P = prolong(chc).tocsc()
    nvf, nvc = 2 * 4 * chc.Nx * chc.Ny, 2 * chc.Nx * chc.Ny
    Rv = 0.25 * P[:nvf, :nvc].T
    rows, cols, vals = [], [], []
    for J in range(chc.Ny):
        for I in range(chc.Nx):
            for b in (0, 1):
                for a in (0, 1):
                    rows.append(J * chc.Nx + I)
                    cols.append((2 * J + b) * (2 * chc.Nx) + 2 * I + a)
                    vals.append(0.25)
    Rp = sp.csr_matrix((vals, (rows, cols)), shape=(chc.Nx * chc.Ny, 4 * chc.Nx * chc.Ny))
    return sp.block_diag([Rv, Rp], format="csr")


def vanka_patches(ch: Channel) -> list:
    """Standard Vanka patches V_ij (Sec. 3.1) of the channel in cell order; the cells next to
    the inflow wall lose their prescribed top face (four unknowns)."""
    out = []
    for j in range(ch.Ny):
        for i in range(ch.Nx):
            d = [ch.iu(i, j), ch.iu(i + 1, j), ch.iv(i, j), ch.ip(i, j)]
            if j + 1 < ch.Ny:
                d.append(ch.iv(i, j + 1))
            out.append(np.array(sorted(set(d)), dtype=np.int64))
    return out


class ChannelLevel:
    def __init__(self, ch: Channel, K: sp.csr_matrix, patches=None, coarsest=False, ee_pattern=None):
        from . import smoother
        self.ch, self.K = ch, K.tocsr()
        self.Kc = self.K.tocsc()
        self.coarsest = coarsest
        self.ee_pattern = ee_pattern  # structural pattern of E_E on this level (velocity block)
        self._colours = None
        if coarsest:
            self.Kinv = np.linalg.inv(self.K.toarray())
        else:
            self.patches = vanka_patches(ch) if patches is None else patches
            self.solvers = [smoother.PatchSolver(self.K, p) for p in self.patches]


def hierarchy(ch: Channel, K: sp.csr_matrix, coarsest_N: int = 8) -> list:
    """Vanka levels from the finest channel (operator K) down to Nx = coarsest_N; coarser
    operators are the rediscretised channel Stokes operator with homogeneous boundary data
    (corrections).  ib_hierarchy below adds a structure's E_E and CAV patches."""
    levels = []
    l = 0
    while True:
        coarsest = ch.Nx // 2 < coarsest_N or ch.Nx % 2 or ch.Ny % 2
        if l > 0:
            K = operator(ch)[0]
        levels.append(ChannelLevel(ch, K, coarsest=coarsest))
        if coarsest:
            return levels
        ch = Channel(ch.Nx // 2, ch.Ny // 2, 2 * ch.h, ch.rho, ch.mu, ch.dt)
        l += 1


def sweep(lev: ChannelLevel, w, b):
    """One multiplicative sweep (Sec. 3.3) in cell order; the channel's pressure is
    determined, so no mean is removed."""
    w = w.copy()
    r = b - lev.K @ w
    for s in lev.solvers:
        d = s.apply(r[s.dofs])
        w[s.dofs] += d
        r -= lev.Kc[:, s.dofs] @ d
    return w


def coupling(lev: ChannelLevel) -> sp.csr_matrix:
    """Structural coupling of the level's K_E: the channel stencil's reach (structure()),
    E_E's pattern in the velocity block, and the diagonal."""
    ch = lev.ch
    pat = sp.csr_matrix(operator(ch, structural=True)[0] != 0, dtype=bool)
    pat = pat + sp.identity(ch.n, dtype=bool, format="csr")
    if lev.ee_pattern is not None:
        nv = 2 * ch.Nx * ch.Ny
        E = sp.csr_matrix(lev.ee_pattern, dtype=bool)
        pat = pat + sp.bmat([[E, None], [None, sp.csr_matrix((ch.n - nv, ch.n - nv), dtype=bool)]],
                            format="csr", dtype=bool)
    pat = sp.csr_matrix(pat, dtype=bool)
    pat.sort_indices()
    return pat


def colours(lev: ChannelLevel) -> np.ndarray:
    """Colour classes of the level's patches for the class-by-class multiplicative sweep:
    first fit over the structural coupling, enlarged patches in cell order, then the standard
    ones (the same relation and order as on the periodic grid, oracle/colouring.py)."""
    from . import colouring
    if lev._colours is None:
        lev._colours = colouring.greedy_colours(lev.patches, coupling(lev))
    return lev._colours


def coloured_sweep(lev: ChannelLevel, w, b):
    """One multiplicative sweep (Sec. 3.3) visiting the colour classes in turn (a class's
    patches in ascending cell order): each patch solves its local residual from the current
    iterate.  No mean is removed."""
    w = np.array(w, dtype=np.float64, copy=True)
    col = colours(lev)
    for k in range(int(col.max()) + 1):
        for c in np.nonzero(col == k)[0]:
            s = lev.solvers[c]
            w[s.dofs] += s.apply(b[s.dofs] - lev.K[s.dofs] @ w)
    return w


def additive_sweep(lev: ChannelLevel, w, b, alpha: float = 1.0):
    """One weighted additive sweep (Eq. additive_cav_saddle) with Theta = 1 / patch count; no
    mean is removed."""
    from . import smoother
    if getattr(lev, "theta", None) is None:
        lev.theta = smoother.partition_weights(lev.patches, lev.ch.n)
    r = b - lev.K @ w
    corr = np.zeros_like(w)
    for s in lev.solvers:
        corr[s.dofs] += lev.theta[s.dofs] * s.apply(r[s.dofs])
    return w + alpha * corr


def _smooth(lev, x, b, mode, alpha):
    if mode == "coloured":
        return coloured_sweep(lev, x, b)
    if mode == "additive":
        return additive_sweep(lev, x, b, alpha)
    return sweep(lev, x, b)


def vcycle(levels, b, nu_pre=1, nu_post=1, li=0, mode="lexicographic", alpha=1.0):
    """z = B b: one V-cycle with zero initial guess on the channel hierarchy (Sec. 4); mode
    "lexicographic" (the paper's multiplicative sweep in cell order), "coloured" (the same
    sweep class by class) or "additive"."""
    lev = levels[li]
    if lev.coarsest:
        return lev.Kinv @ b
    x = np.zeros_like(b)
    for _ in range(nu_pre):
        x = _smooth(lev, x, b, mode, alpha)
    chc = levels[li + 1].ch
    xc = vcycle(levels, restrict(chc) @ (b - lev.K @ x), nu_pre, nu_post, li + 1, mode, alpha)
    x = x + prolong(chc) @ xc
    for _ in range(nu_post):
        x = _smooth(lev, x, b, mode, alpha)
    return x


# --------------------------------------------------------------------------- IB coupling

def cav_patches(ch: Channel, pattern) -> list:
    """CAV patches (Eq. cav_patch_set) on the channel, cell by cell: U^ = U_ij plus every
    velocity coupled to U_ij through E_E's pattern (either direction); if that adds nothing the
    cell keeps its Vanka patch, else the patch is the union of the Vanka patches of the cells
    incident to U^ -- a u face's two neighbouring cells, a v face's cells below and above, the
    outflow row's faces having only the cell above."""
    Nx, Ny = ch.Nx, ch.Ny
    NN = Nx * Ny
    Pr = sp.csr_matrix(pattern, dtype=bool)
    Pc = Pr.T.tocsr()
    van = vanka_patches(ch)
    out = []
    for c in range(NN):
        U = [int(k) for k in van[c] if k < 2 * NN]
        Uh = set(U)
        for k in U:
            Uh.update(int(l) for l in Pr.indices[Pr.indptr[k]:Pr.indptr[k + 1]])
            Uh.update(int(l) for l in Pc.indices[Pc.indptr[k]:Pc.indptr[k + 1]])
        if Uh == set(U):
            out.append(van[c])
            continue
        cells = set()
        for k in Uh:
            comp, rem = divmod(k, NN)
            j, i = divmod(rem, Nx)
            if comp == 0:
                cells.update({j * Nx + (i - 1) % Nx, j * Nx + i})
            else:
                cells.add(j * Nx + i)
                if j >= 1:
                    cells.add((j - 1) * Nx + i)
        out.append(np.array(sorted(set().union(*(set(van[q].tolist()) for q in cells))), dtype=np.int64))
    return out


def galerkin_elasticity(EE_f: sp.csr_matrix, chc: Channel) -> sp.csr_matrix:
    """E_E on the coarse channel: R_v E_E P_v with the channel's velocity transfers (Sec. 4)."""
    P = prolong(chc).tocsc()
    nvf, nvc = 2 * 4 * chc.Nx * chc.Ny, 2 * chc.Nx * chc.Ny
    Pv = P[:nvf, :nvc]
    return (0.25 * Pv.T @ EE_f @ Pv).tocsr()


def ib_hierarchy(ch: Channel, EE: sp.csr_matrix, pattern, coarsest_N: int = 8):
    """The finest operator K_E = K0 - dt [[E_E, 0], [0, 0]] and its CAV hierarchy on the
    channel: Galerkin E_E and structural patterns level by level, CAV patches from them."""
    levels = []
    c, EEl, patl = ch, EE.tocsr(), sp.csr_matrix(pattern, dtype=bool)
    while True:
        nv = 2 * c.Nx * c.Ny
        K = (operator(c)[0] - c.dt * sp.bmat([[EEl, None], [None, sp.csr_matrix((c.n - nv, c.n - nv))]])).tocsr()
        coarsest = c.Nx // 2 < coarsest_N or c.Nx % 2 or c.Ny % 2
        levels.append(ChannelLevel(c, K, patches=None if coarsest else cav_patches(c, patl), coarsest=coarsest,
                                   ee_pattern=patl))
        if coarsest:
            return levels
        cc = Channel(c.Nx // 2, c.Ny // 2, 2 * c.h, c.rho, c.mu, c.dt)
        EEl = galerkin_elasticity(EEl, cc)
        Pv = prolong(cc).tocsc()[:2 * 4 * cc.Nx * cc.Ny, :2 * cc.Nx * cc.Ny]
        Pb = sp.csr_matrix(Pv != 0, dtype=np.float64)
        patl = sp.csr_matrix((Pb.T @ sp.csr_matrix(patl, dtype=np.float64) @ Pb) != 0, dtype=bool)
        c = cc


# --------------------------------------------------------------------------- time step (Sec. 5.3)

def inflow_speed(t: float, U: float = 1.0, T_ramp: float = 0.5625) -> float:
    """Magnitude of the downward inflow at time t: raised smoothly from 0 to U over [0, T_ramp]
    (the paper says "smoothly"; the reading is the half-cosine ramp U (1 - cos(pi t / T)) / 2)."""
    if t >= T_ramp:
        return U
    return U * 0.5 * (1.0 - np.cos(np.pi * t / T_ramp))


def _ghosts(ch: Channel, w, u_top, v_top, t_x):
    """Padded velocity arrays with the boundary ghosts of the operator: u (Ny + 2, Nx) over rows
    -1 .. Ny, v (Ny + 2, Nx) over rows -1 .. Ny (row Ny prescribed)."""
    Nx, Ny, h, mu = ch.Nx, ch.Ny, ch.h, ch.mu
    NN = Nx * Ny
    u = w[:NN].reshape(Ny, Nx)
    v = w[NN:2 * NN].reshape(Ny, Nx)
    U = np.zeros((Ny + 2, Nx))
    V = np.zeros((Ny + 2, Nx))
    U[1:Ny + 1] = u
    U[Ny + 1] = 2.0 * u_top - u[Ny - 1]
    U[0] = u[0] + (v[0] - np.roll(v[0], 1)) + h * t_x / mu
    V[1:Ny + 1] = v
    V[Ny + 1] = v_top
    V[0] = v[0] + (np.roll(U[0], -1) - U[0])
    return U, V


def convection(ch: Channel, w, u_top=0.0, v_top=None, t_x=None) -> np.ndarray:
    """N[u] = (u . grad) u on the velocity faces (2 Nx Ny), centred differences, each
    component averaged from its four neighbours onto the other's faces (Sec. 2's explicit
    convective term); boundary values through the operator's ghosts."""
    Nx, Ny, h = ch.Nx, ch.Ny, ch.h
    v_top = np.zeros(Nx) if v_top is None else np.asarray(v_top, dtype=np.float64)
    t_x = np.zeros(Nx) if t_x is None else np.asarray(t_x, dtype=np.float64)
    U, V = _ghosts(ch, w, u_top, v_top, t_x)
    # u faces (rows 0 .. Ny-1 = padded 1 .. Ny)
    u = U[1:Ny + 1]
    dudx = (np.roll(u, -1, 1) - np.roll(u, 1, 1)) / (2 * h)
    dudy = (U[2:Ny + 2] - U[0:Ny]) / (2 * h)
    vbar = 0.25 * (V[1:Ny + 1] + np.roll(V[1:Ny + 1], 1, 1) + V[2:Ny + 2] + np.roll(V[2:Ny + 2], 1, 1))
    Nu = u * dudx + vbar * dudy
    # v faces (rows 0 .. Ny-1)
    v = V[1:Ny + 1]
    dvdx = (np.roll(v, -1, 1) - np.roll(v, 1, 1)) / (2 * h)
    dvdy = (V[2:Ny + 2] - V[0:Ny]) / (2 * h)
    ubar = 0.25 * (U[1:Ny + 1] + np.roll(U[1:Ny + 1], -1, 1) + U[0:Ny] + np.roll(U[0:Ny], -1, 1))
    Nv = ubar * dvdx + v * dvdy
    return np.concatenate([Nu.ravel(), Nv.ravel()])


def backflow_traction(ch: Channel, w):
    """t = (rho/2) min(u.n, 0) u at the outflow y = 0, n = (0, -1), from the velocity w (the
    previous step's): t_x at the points (i h, 0), t_y at ((i + 1/2) h, 0).  The boundary u is
    extrapolated from the first two rows, (3 u_0 - u_1)/2; v at (i h, 0) is the mean of its
    two neighbours."""
    Nx, Ny = ch.Nx, ch.Ny
    NN = Nx * Ny
    u = w[:NN].reshape(Ny, Nx)
    v = w[NN:2 * NN].reshape(Ny, Nx)
    ub = 0.5 * (3.0 * u[0] - u[1])
    vb_u = 0.5 * (v[0] + np.roll(v[0], 1))        # v at (i h, 0)
    ub_v = 0.5 * (ub + np.roll(ub, -1))           # u at ((i + 1/2) h, 0)
    t_x = 0.5 * ch.rho * np.minimum(-vb_u, 0.0) * ub
    t_y = 0.5 * ch.rho * np.minimum(-v[0], 0.0) * v[0]
    return t_x, t_y


def fiber_step(ch: Channel, rec, w_n, t_next: float, solver: str = "direct", rtol=1e-8, atol=1e-8,
               maxit=20, fgmres_rtol=1e-9, mode: str = "lexicographic"):
    """One time step of Sec. 5.3's scheme in the channel, from the velocity-pressure w_n at t^n
    and the fiber configuration rec.X = X^n to t^{n+1} = t_next:

        rho/dt (u - u^n) + rho N[u^n] - mu L u + G p = S^n F(X^n + dt J^n u),   -D u = 0,

    the inflow v = -U(t^{n+1}) on the top wall, the traction outflow with the backflow term at
    u^n, the convective term explicit at u^n.  Newton's method on (u, p) (oracle/newton.py's
    iteration) with each linear system solved directly ("direct") or by CAV-preconditioned
    FGMRES with the hierarchy rebuilt per Newton system ("cav", 1 + 1 sweeps of the given mode,
    as the paper does).  The FGMRES solve of Newton system k starts from the iterate w_k and
    stops at fgmres_rtol relative to its initial residual, which is the Newton residual at w_k:
    an inexact Newton step whose forcing term is fgmres_rtol (reading: the paper's 1e-9 for
    FGMRES and 1e-8 for Newton both relative to the current residual; a zero initial guess
    with the tolerance relative to the whole right-hand side caps the Newton residual at
    fgmres_rtol ||rhs||, and Newton stalls once the flow settles).  Returns (w, X^{n+1},
    residual history, FGMRES counts)."""
    from dataclasses import replace

    import scipy.sparse.linalg as spla

    from . import fgmres, ib
    Nx = ch.Nx
    NN2 = 2 * Nx * ch.Ny
    S = ib.spreading_matrix(rec.N, rec.h, rec.X, rec.omega)
    J = ib.interpolation_matrix(rec.N, rec.h, rec.X)
    Xn = np.concatenate([rec.X[:, 0], rec.X[:, 1]])
    M = rec.M
    v_top_n = np.full(Nx, -inflow_speed(t_next - ch.dt))
    v_top = np.full(Nx, -inflow_speed(t_next))
    t_x, t_y = backflow_traction(ch, w_n)
    K0, g = operator(ch, 0.0, v_top, t_x, t_y)
    b = np.zeros(ch.n)
    b[:NN2] = ch.rho / ch.dt * w_n[:NN2] - ch.rho * convection(ch, w_n, 0.0, v_top_n, t_x)
    b += g

    def force_at(u):
        Xk = Xn + ch.dt * (J @ u)
        rk = replace(rec, meta={**rec.meta, "X_lin": np.stack([Xk[:M], Xk[M:]], 1)})
        return rk, ib.force_vector(rk)

    def residual(w):
        _, F = force_at(w[:NN2])
        R = K0 @ w - b
        R[:NN2] -= S @ F
        return R

    w = np.array(w_n, dtype=np.float64)
    hist = [np.linalg.norm(residual(w))]
    its = []
    k = 0
    while k < maxit and hist[-1] > max(rtol * hist[0], atol):
        rk, F = force_at(w[:NN2])
        EE, pat = ib.eulerian_elasticity(rk)
        E, _ = ib.elasticity(rk)
        K = (K0 - ch.dt * sp.bmat([[EE, None], [None, sp.csr_matrix((ch.n - NN2, ch.n - NN2))]])).tocsr()
        rhs = b.copy()
        rhs[:NN2] += S @ (F - ch.dt * (E @ (J @ w[:NN2])))
        if solver == "direct":
            w = spla.spsolve(K.tocsc(), rhs)
        else:
            levels = ib_hierarchy(ch, EE, pat)
            w, info = fgmres.fgmres(lambda v: K @ v, rhs, lambda r: vcycle(levels, r, mode=mode), x0=w,
                                    rtol=fgmres_rtol, maxit=150, ref="r0")
            its.append(info["iters"])
        k += 1
        hist.append(np.linalg.norm(residual(w)))
    X_next = Xn + ch.dt * (J @ w[:NN2])
    return w, np.stack([X_next[:M], X_next[M:]], 1), hist, its
