"""Hand-built inputs for pin tests (tiny networks with chosen parameters)."""
import numpy as np

from paper_2512_06729_gb300 import synth


def nasa_const_cp(a1, a6, a7, tmid=1000.0):
    """NASA-7 set with constant C_p/R = a1 (a2..a5 = 0), same in both ranges."""
    row = np.zeros(15)
    row[0] = tmid
    for base in (1, 8):
        row[base + 0] = a1
        row[base + 5] = a6
        row[base + 6] = a7
    return row


def custom_problem(elem, mass, reactions, nasa, P_bar, T, Kzz=None, dcoef=None, f0=None,
                   photo=None, g=2.0e3, mbar=2.3, alpha_T=0.0, mu=0.5, tf=0.5, name="custom"):
    """reactions: list of dicts with keys type (0/1/2), reac, prod, arr (9), troe (4), form."""
    elem = np.asarray(elem, np.int32)
    S = elem.shape[0]
    P_bar = np.atleast_1d(np.asarray(P_bar, float))
    T = np.atleast_1d(np.asarray(T, float))
    L = P_bar.shape[0]
    R = len(reactions)
    rtype = np.zeros(R, np.int32); reac = -np.ones((R, 3), np.int32); prod = -np.ones((R, 3), np.int32)
    arr = np.zeros((R, 9)); troe = np.zeros((R, 4)); form = np.zeros(R, np.int32)
    for i, rx in enumerate(reactions):
        rtype[i] = rx["type"]
        reac[i, : len(rx["reac"])] = rx["reac"]
        prod[i, : len(rx["prod"])] = rx["prod"]
        arr[i, : len(rx.get("arr", []))] = rx.get("arr", [])
        troe[i, : len(rx.get("troe", []))] = rx.get("troe", [])
        form[i] = rx.get("form", 0)
    prow = -np.ones(R, np.int32)
    ph = np.flatnonzero(rtype == 2)
    prow[ph] = np.arange(len(ph))
    if photo is None:
        lam = np.zeros(0); dlam = np.zeros(0); J0 = np.zeros(0)
        sigma = np.zeros((len(ph), 0)); sigma_abs = np.zeros((S, 0))
    else:
        lam, dlam, J0, sigma, sigma_abs = photo
    return synth.Problem(
        name=name, elements=[f"e{i}" for i in range(elem.shape[1])], elem=elem,
        mass=np.asarray(mass, float), rtype=rtype, reac=reac, prod=prod, arr=arr, troe=troe,
        form=form, nasa=np.asarray(nasa, float), prow=prow, lam=lam, dlam=dlam, J0=J0,
        sigma=sigma, sigma_abs=sigma_abs, mu=mu, tf=tf, P_bar=P_bar, T=T,
        Kzz=np.zeros(L) if Kzz is None else np.asarray(Kzz, float),
        dcoef=np.zeros(S) if dcoef is None else np.asarray(dcoef, float),
        g=g, mbar=mbar, alpha_T=alpha_T,
        f0=np.full((L, S), 1.0 / S) if f0 is None else np.asarray(f0, float))


def read_nasa_table(path):
    sets = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        parts = line.split()
        name, rng = parts[0], parts[1]
        sets.setdefault(name, {})[rng] = [float(x) for x in parts[2:9]]
    out = {}
    for name, d in sets.items():
        row = np.zeros(15)
        row[0] = 1000.0
        row[1:8] = d["low"]
        row[8:15] = d["high"]
        out[name] = row
    return out


def full_matrix(A, lo, up):
    L, S = lo.shape
    M = np.zeros((L * S, L * S))
    for k in range(L):
        M[k * S:(k + 1) * S, k * S:(k + 1) * S] = A[k]
        if k > 0:
            M[k * S:(k + 1) * S, (k - 1) * S:k * S] = np.diag(lo[k])
        if k < L - 1:
            M[k * S:(k + 1) * S, (k + 1) * S:(k + 2) * S] = np.diag(up[k])
    return M


def independent_block_solve(A, lo, up, f):
    """A second FP64 solve of the block-tridiagonal system, independent of the
    oracle's own LU: block Thomas on LAPACK's blocked partial-pivot LU
    (scipy.linalg.lu_factor / lu_solve), whose rounding differs from the
    oracle's column-by-column elimination.  The difference between the two is
    the accuracy FP64 itself reaches on the system, the yardstick of the
    parity bounds."""
    from scipy.linalg import lu_factor, lu_solve
    L, S = lo.shape
    lus, g = [], np.array(f, dtype=np.float64, copy=True)
    for k in range(L):
        D = np.array(A[k], dtype=np.float64, copy=True)
        if k > 0:
            D -= lo[k][:, None] * lu_solve(lus[k - 1], np.diag(up[k - 1]))
            g[k] -= lo[k] * lu_solve(lus[k - 1], g[k - 1])
        lus.append(lu_factor(D, check_finite=False))
    x = np.empty_like(g)
    for k in range(L - 1, -1, -1):
        rhs = g[k] - (up[k] * x[k + 1] if k + 1 < L else 0.0)
        x[k] = lu_solve(lus[k], rhs)
    return x


def relative_to_state(d, ref, n, ngas, floor=1e-20):
    """Largest |d - ref| / n over the entries above floor mixing ratio."""
    keep = n > floor * ngas[:, None]
    return float(np.max(np.abs(d - ref)[keep] / n[keep])) if keep.any() else 0.0


def independent_refined_solve(A, lo, up, f, s, sweeps=4):
    """The step's linear system solved a second way, independent of the
    oracle's code: in relative variables y = x / s (diag(1/s) A diag(s) y =
    f / s), block Thomas on LAPACK's LU, then FP64 iterative refinement on the
    scaled system.  Returns x."""
    from scipy.linalg import lu_factor, lu_solve
    L, S = lo.shape
    As = A * s[:, None, :] / s[:, :, None]
    los = np.zeros_like(lo); los[1:] = lo[1:] * s[:-1] / s[1:]
    ups = np.zeros_like(up); ups[:-1] = up[:-1] * s[1:] / s[:-1]
    b = f / s
    lus = []
    for k in range(L):
        D = As[k].copy()
        if k > 0:
            D -= los[k][:, None] * lu_solve(lus[k - 1], np.diag(ups[k - 1]))
        lus.append(lu_factor(D, check_finite=False))

    def apply(r):
        g = r.copy()
        for k in range(1, L):
            g[k] -= los[k] * lu_solve(lus[k - 1], g[k - 1])
        y = np.empty_like(g)
        for k in range(L - 1, -1, -1):
            y[k] = lu_solve(lus[k], g[k] - (ups[k] * y[k + 1] if k + 1 < L else 0.0))
        return y

    def matvec(y):
        r = np.einsum("kij,kj->ki", As, y)
        r[1:] += los[1:] * y[:-1]
        r[:-1] += ups[:-1] * y[1:]
        return r

    y = apply(b)
    for _ in range(sweeps):
        y = y + apply(b - matvec(y))
    return y * s
