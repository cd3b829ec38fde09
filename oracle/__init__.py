"""CPU oracle for mixed-precision iterative refinement of LSE / GLS problems.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product library (``paper_2406_16499_gb300``) never
imports it and shares no code with it.

Everything here is a thin ctypes layer over ``mpir_oracle.c`` (plain C, FP64,
unblocked Householder, double-double residuals) plus small numpy helpers for
norms and error metrics.  Each function names the part of the paper it
follows:

* ``lse_solve`` / ``gls_solve``        -- Alg. 2 (MPLSE) / Alg. 4 (MPGLS)
* ``lse_residual`` / ``gls_residual``  -- residuals of eq. aug-LSE / aug-GLS
* ``lse_factor`` / ``gls_factor``      -- GRQ / GQR (Sec. 2, Lemma 4.5/4.6)
* ``lse_correction`` / ``gls_correction`` -- Alg. 1 / Alg. 3
* ``lse_truth`` / ``gls_truth``        -- FP64 factors + double-double
  residual refinement: the exact solution up to ~u (Table 2, u_r = quad row)
* ``lse_metrics`` / ``gls_metrics``    -- eq. lse-stop / gls-stop ratios,
  err-1 of Tables 4 and 5
* ``lse_kappa`` / ``gls_kappa``        -- condition numbers for the
  forward-error tolerance (power iteration on FP64 factors)

``oracle/gmres.py`` restates GMRES-IR (Sec. 5), ``oracle/selector.py`` the
selector, and ``oracle/zoracle.py`` the complex problems (Sec. 1 defines both
over C) with dense numpy factors.

All pins that tie these functions to the paper and to independent
mathematics are in ``tests/test_oracle_*.py``.
"""
import ctypes
import numpy as np

from . import build as _build

_c_int = ctypes.c_int
_c_dbl = ctypes.c_double
_P = ctypes.POINTER(ctypes.c_double)
_PI = ctypes.POINTER(ctypes.c_int)

_lib = None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        I, D = _c_int, _c_dbl
        L.or_lse_solve.argtypes = [I, I, I, _P, I, _P, I, _P, _P, _P, _P, _P, I, I, D, I, _PI, _P]
        L.or_gls_solve.argtypes = [I, I, I, _P, I, _P, I, _P, _P, _P, _P, I, I, D, I, _PI, _P]
        L.or_lse_residual.argtypes = [I, I, I, _P, I, _P, I, _P, _P, _P, _P, _P, _P, _P, _P, I]
        L.or_gls_residual.argtypes = [I, I, I, _P, I, _P, I, _P, _P, _P, _P, _P, _P, _P, I]
        L.or_lse_factor.argtypes = [I, I, I, _P, I, _P, I, I, _P, _P, _P, _P]
        L.or_gls_factor.argtypes = [I, I, I, _P, I, _P, I, I, _P, _P, _P, _P]
        L.or_lse_apply.argtypes = [I, I, I, _P, _P, _P, _P, I, I, _P]
        L.or_gls_apply.argtypes = [I, I, I, _P, _P, _P, _P, I, I, _P]
        L.or_lse_nullspace.argtypes = [I, I, I, _P, _P, _P, _P, _P, _P, _P]
        L.or_gls_paige.argtypes = [I, I, I, _P, _P, _P, _P, _P, _P, _P]
        L.or_lse_correction.argtypes = [I, I, I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]
        L.or_gls_correction.argtypes = [I, I, I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]
        L.or_lse_init_v.argtypes = [I, I, I, _P, _P, _P, _P, _P, I, _P, _P]
        L.or_gls_init_z.argtypes = [I, I, I, _P, _P, _P, _P, _P, _P]
        L.or_lse_kappa.argtypes = [I, I, I, _P, _P, _P, _P, I, _P]
        L.or_gls_kappa.argtypes = [I, I, I, _P, _P, _P, _P, I, _P]
        for f in ("or_lse_solve", "or_gls_solve", "or_num_threads"):
            getattr(L, f).restype = _c_int
        _lib = L
    return _lib


def num_threads():
    return int(lib().or_num_threads())


def _F(a):
    """Column-major float64 copy-or-view (the oracle reads column-major)."""
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _v(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel())


def _p(a):
    if a.size == 0:
        a = np.zeros(1)
    return a.ctypes.data_as(_P)


def _ld(a, rows):
    return max(1, rows)


# ---------------------------------------------------------------- solves --

def lse_solve(A, B, b, d, fact="fp64", maxit=40, tol=2e-15, resid_dd=False):
    """Alg. 2 (MPLSE).  fact: 'fp64' or 'fp32' (u_f = u_s).  Residuals in
    FP64 (u_r = u), or double-double with resid_dd.  Returns a dict with
    x, r, v, status (0 ok, 3 maxit, 4 non-finite), iters, ratios."""
    A, B = _F(A), _F(B)
    m, n = A.shape
    p = B.shape[0]
    b, d = _v(b), _v(d)
    x, r, v = np.zeros(n), np.zeros(m), np.zeros(p)
    it = ctypes.c_int(0)
    ratios = np.zeros(3)
    st = lib().or_lse_solve(m, n, p, _p(A), _ld(A, m), _p(B), _ld(B, p), _p(b), _p(d),
                            _p(x), _p(r), _p(v), 1 if fact == "fp32" else 0, maxit, tol,
                            1 if resid_dd else 0, ctypes.byref(it), _p(ratios))
    return dict(x=x, r=r, v=v, status=st, iters=it.value, ratios=ratios)


def gls_solve(W, V, d, fact="fp64", maxit=40, tol=2e-15, resid_dd=False):
    """Alg. 4 (MPGLS).  Same conventions as lse_solve; returns x, y, z."""
    W, V = _F(W), _F(V)
    n, m = W.shape
    p = V.shape[1]
    d = _v(d)
    x, y, z = np.zeros(m), np.zeros(p), np.zeros(n)
    it = ctypes.c_int(0)
    ratios = np.zeros(3)
    st = lib().or_gls_solve(n, m, p, _p(W), _ld(W, n), _p(V), _ld(V, n), _p(d), _p(x), _p(y),
                            _p(z), 1 if fact == "fp32" else 0, maxit, tol,
                            1 if resid_dd else 0, ctypes.byref(it), _p(ratios))
    return dict(x=x, y=y, z=z, status=st, iters=it.value, ratios=ratios)


def lse_truth(A, B, b, d, steps=3):
    """The LSE solution to ~u: FP64 GRQ, null-space start, `steps`
    refinement steps with double-double residuals (Table 2, u_r = quad)."""
    return lse_solve(A, B, b, d, fact="fp64", maxit=steps, tol=0.0, resid_dd=True)


def gls_truth(W, V, d, steps=3):
    """The GLS solution (x, minimum-norm y, z) to ~u, as lse_truth."""
    return gls_solve(W, V, d, fact="fp64", maxit=steps, tol=0.0, resid_dd=True)


# ------------------------------------------------------------- residuals --

def lse_residual(A, B, b, d, x, r, v, dd=True):
    """f1 = b - r - A x, f2 = d - B x, f3 = -A^T r + B^T v (eq. aug-LSE)."""
    A, B = _F(A), _F(B)
    m, n = A.shape
    p = B.shape[0]
    f1, f2, f3 = np.zeros(m), np.zeros(p), np.zeros(n)
    lib().or_lse_residual(m, n, p, _p(A), _ld(A, m), _p(B), _ld(B, p), _p(_v(b)), _p(_v(d)),
                          _p(_v(x)), _p(_v(r)), _p(_v(v)), _p(f1), _p(f2), _p(f3),
                          1 if dd else 0)
    return f1, f2, f3


def gls_residual(W, V, d, x, y, z, dd=True):
    """f1 = -y + V^T z, f2 = d - W x - V y, f3 = W^T z (eq. aug-GLS)."""
    W, V = _F(W), _F(V)
    n, m = W.shape
    p = V.shape[1]
    f1, f2, f3 = np.zeros(p), np.zeros(n), np.zeros(m)
    lib().or_gls_residual(n, m, p, _p(W), _ld(W, n), _p(V), _ld(V, n), _p(_v(d)), _p(_v(x)),
                          _p(_v(y)), _p(_v(z)), _p(f1), _p(f2), _p(f3), 1 if dd else 0)
    return f1, f2, f3


# --------------------------------------------------------------- factors --

def lse_factor(A, B, fact="fp64"):
    """Packed GRQ factors of (B, A): RQ of B in Bf/taub (row reflectors,
    R in Bf[:, n-p:]), QR of A Q^T in Af/taua (T in the upper trapezoid)."""
    A, B = _F(A), _F(B)
    m, n = A.shape
    p = B.shape[0]
    Bf, Af = np.zeros((p, n), order="F"), np.zeros((m, n), order="F")
    taub, taua = np.zeros(max(p, 1)), np.zeros(max(min(m, n), 1))
    lib().or_lse_factor(m, n, p, _p(A), _ld(A, m), _p(B), _ld(B, p), 1 if fact == "fp32" else 0,
                        _p(Bf), _p(taub), _p(Af), _p(taua))
    return dict(kind="lse", m=m, n=n, p=p, Bf=Bf, taub=taub, Af=Af, taua=taua)


def gls_factor(W, V, fact="fp64"):
    """Packed GQR factors of (W, V): QR of W in Wf/tauw (R in Wf[:m]), RQ of
    Q^T V in Vf/tauv (T in the upper trapezoid, RQ sense)."""
    W, V = _F(W), _F(V)
    n, m = W.shape
    p = V.shape[1]
    Wf, Vf = np.zeros((n, m), order="F"), np.zeros((n, p), order="F")
    tauw, tauv = np.zeros(max(m, 1)), np.zeros(max(min(n, p), 1))
    lib().or_gls_factor(n, m, p, _p(W), _ld(W, n), _p(V), _ld(V, n), 1 if fact == "fp32" else 0,
                        _p(Wf), _p(tauw), _p(Vf), _p(tauv))
    return dict(kind="gls", n=n, m=m, p=p, Wf=Wf, tauw=tauw, Vf=Vf, tauv=tauv)


def _fargs(F):
    if F["kind"] == "lse":
        return (F["m"], F["n"], F["p"], _p(F["Bf"]), _p(F["taub"]), _p(F["Af"]), _p(F["taua"]))
    return (F["n"], F["m"], F["p"], _p(F["Wf"]), _p(F["tauw"]), _p(F["Vf"]), _p(F["tauv"]))


def apply(F, which, x, trans=False):
    """Apply a factor's orthogonal matrix to vector x (returns a copy).
    which: 'Q' or 'Z' (the paper's names for the problem kind of F)."""
    x = _v(x).copy()
    fn = lib().or_lse_apply if F["kind"] == "lse" else lib().or_gls_apply
    fn(*_fargs(F), 0 if which == "Q" else 1, 1 if trans else 0, _p(x))
    return x


def explicit(F, which):
    """Dense orthogonal factor (columns = images of unit vectors)."""
    if F["kind"] == "lse":
        k = F["n"] if which == "Q" else F["m"]
    else:
        k = F["n"] if which == "Q" else F["p"]
    I = np.eye(k)
    return np.column_stack([apply(F, which, I[:, j]) for j in range(k)])


def R_T(F):
    """(R, T) as dense arrays with the reflector storage zeroed."""
    if F["kind"] == "lse":
        m, n, p = F["m"], F["n"], F["p"]
        R = np.triu(F["Bf"][:, n - p:])
        T = np.triu(F["Af"])
        return R, T
    n, m, p = F["n"], F["m"], F["p"]
    R = np.triu(F["Wf"][:m, :])
    k = min(n, p)
    T = F["Vf"].copy()
    for r in range(n - k, n):
        T[r, : max(0, p - n + r)] = 0.0
    return R, T


def lse_nullspace(F, b, d):
    x = np.zeros(F["n"])
    lib().or_lse_nullspace(*_fargs(F), _p(_v(b)), _p(_v(d)), _p(x))
    return x


def gls_paige(F, d):
    x, y = np.zeros(F["m"]), np.zeros(F["p"])
    lib().or_gls_paige(*_fargs(F), _p(_v(d)), _p(x), _p(y))
    return x, y


def lse_init_v(F, A, r):
    A = _F(A)
    v = np.zeros(F["p"])
    lib().or_lse_init_v(*_fargs(F), _p(A), _ld(A, F["m"]), _p(_v(r)), _p(v))
    return v


def gls_init_z(F, y):
    z = np.zeros(F["n"])
    lib().or_gls_init_z(*_fargs(F), _p(_v(y)), _p(z))
    return z


def lse_correction(F, f1, f2, f3):
    """Alg. 1 in FP64 on the given factors -> (dr, dv, dx)."""
    dr, dv, dx = np.zeros(F["m"]), np.zeros(F["p"]), np.zeros(F["n"])
    lib().or_lse_correction(*_fargs(F), _p(_v(f1)), _p(_v(f2)), _p(_v(f3)),
                            _p(dr), _p(dv), _p(dx))
    return dr, dv, dx


def gls_correction(F, f1, f2, f3):
    """Alg. 3 (readings: T22 g2 = u2, dz = -Q h) in FP64 -> (dy, dz, dx)."""
    dy, dz, dx = np.zeros(F["p"]), np.zeros(F["n"]), np.zeros(F["m"])
    lib().or_gls_correction(*_fargs(F), _p(_v(f1)), _p(_v(f2)), _p(_v(f3)),
                            _p(dy), _p(dz), _p(dx))
    return dy, dz, dx


# --------------------------------------------------------------- metrics --

def lse_metrics(A, B, b, d, x, r, v):
    """Backward-error ratios of eq. lse-stop with double-double residuals
    (eta = their max) and err-1 of Table 4: ||Bx-d||/(||B||_F||x||+||d||)."""
    f1, f2, f3 = lse_residual(A, B, b, d, x, r, v, dd=True)
    nA, nB = np.linalg.norm(A), np.linalg.norm(B)
    nx, nr, nv = np.linalg.norm(x), np.linalg.norm(r), np.linalg.norm(v)
    d1 = np.linalg.norm(b) + nr + nA * nx
    d2 = np.linalg.norm(d) + nB * nx
    d3 = nA * nr + nB * nv
    rat = [np.linalg.norm(f1) / d1 if d1 else 0.0,
           np.linalg.norm(f2) / d2 if d2 else 0.0,
           np.linalg.norm(f3) / d3 if d3 else 0.0]
    e_con = np.linalg.norm(f2) / d2 if d2 else 0.0
    return dict(ratios=rat, eta=max(rat), e_con=e_con)


def gls_metrics(W, V, d, x, y, z):
    """Ratios of eq. gls-stop (double-double residuals) and err-1 of
    Table 5: ||Wx+Vy-d||/(||W||_F||x||+||V||_F||y||+||d||)."""
    f1, f2, f3 = gls_residual(W, V, d, x, y, z, dd=True)
    nW, nV = np.linalg.norm(W), np.linalg.norm(V)
    nx, ny, nz = np.linalg.norm(x), np.linalg.norm(y), np.linalg.norm(z)
    d1 = ny + nV * nz
    d2 = np.linalg.norm(d) + nW * nx + nV * ny
    d3 = nW * nz
    rat = [np.linalg.norm(f1) / d1 if d1 else 0.0,
           np.linalg.norm(f2) / d2 if d2 else 0.0,
           np.linalg.norm(f3) / d3 if d3 else 0.0]
    return dict(ratios=rat, eta=max(rat), e_con=rat[1])


def lse_kappa(F, x, r, iters=60):
    """[kappa, kappa2(T11), kappa2(R)] estimated from FP64 factors."""
    out = np.zeros(3)
    lib().or_lse_kappa(F["m"], F["n"], F["p"], _p(F["Bf"]), _p(F["Af"]), _p(_v(x)), _p(_v(r)),
                       iters, _p(out))
    return out


def gls_kappa(F, x, y, iters=60):
    """[kappa, kappa2(S^{-1} R)] estimated from FP64 factors (n <= p)."""
    out = np.zeros(2)
    lib().or_gls_kappa(F["n"], F["m"], F["p"], _p(F["Wf"]), _p(F["Vf"]), _p(_v(x)), _p(_v(y)),
                       iters, _p(out))
    return out


def forward_error(x, x_ref):
    nref = np.linalg.norm(x_ref)
    return np.linalg.norm(np.asarray(x) - x_ref) / (nref if nref else 1.0)
