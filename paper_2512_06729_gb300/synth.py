"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws inputs only: species element vectors, reaction lists and
their rate parameters, NASA-7 coefficient sets, cross sections, a stellar
spectrum, pressure-temperature-Kzz profiles and initial mixing ratios.  It
evaluates no part of the photochemical method (no rate law, no Gibbs energy,
no grid, no transport, no solver), so that the CUDA path and the CPU oracle
both start from the same raw arrays and compute everything else on their own.

The paper's networks (XODIAC-2025: 594 species / 7,720 reactions, Sec. 2.2),
cross-section databases and stellar spectra are not public; the generators
below stand in for them with the same sizes and the same structure:
element-balanced two-body reactions (Sec. 2.3.1), three-body association
reactions with fall-off (Sec. 2.3.2), photodissociations A -> B + C
(Sec. 2.3.3), NASA-7 polynomials in two temperature ranges (Appendix A),
log-spaced pressure grids with a hot-Jupiter-like temperature profile (Fig. 3).
"""
from __future__ import annotations

import dataclasses
import numpy as np

# Element symbols and atomic masses (u).
ELEMENT_MASS = {
    "H": 1.008, "He": 4.0026, "C": 12.011, "N": 14.007, "O": 15.999,
    "P": 30.974, "S": 32.06, "Na": 22.990, "K": 39.098, "Fe": 55.845,
    "Mg": 24.305, "Si": 28.085, "Ti": 47.867, "Cl": 35.45,
}

RX_TWO_BODY = 0
RX_THREE_BODY = 1
RX_PHOTO = 2

FORM_KOOIJ = 0
FORM_ARRHENIUS = 1


@dataclasses.dataclass
class Problem:
    """All raw inputs of one atmospheric column (host numpy arrays).

    Layout (row-major, C order):
      elem[S, E] int32   element counts per species
      mass[S]            molecular mass (u)
      rtype[R] int32     0 two-body, 1 three-body (fall-off), 2 photolysis
      reac[R, 3], prod[R, 3] int32 species indices, -1 padded
      arr[R, 9]          alpha, beta, gamma | alpha0, beta0, gamma0 | alpha_inf, beta_inf, gamma_inf
      troe[R, 4]         a, T***, T*, T** (a == 0: plain Lindemann)
      form[R] int32      0 Kooij (T_b = T/300), 1 modified Arrhenius (T_b = T)
      nasa[S, 15]        T_mid, a1..a7 (low range), a1..a7 (high range)
      prow[R] int32      row of sigma for a photolysis reaction, else -1
      lam[W], dlam[W]    bin centres and widths (Angstrom)
      J0[W]              top-of-atmosphere photon flux (photons cm^-2 s^-1 A^-1)
      sigma[Rph, W]      photodissociation cross sections (cm^2)
      sigma_abs[S, W]    absorption cross sections used for the optical depth (cm^2)
      P_bar[L], T[L], Kzz[L]   layer pressure (bar), temperature (K), eddy coefficient (cm^2/s)
      dcoef[S]           molecular-diffusion coefficient b_y in D_y = b_y T^0.75 / n_gas
      f0[L, S]           initial mixing ratios
      sigma_s[S, W]      Rayleigh scattering cross sections (None: no scattering)
      albedo, diffuse    lower-boundary albedo; 1 adds the diffuse field to the direct beam
    Layer 0 is the bottom of the atmosphere.
    """

    name: str
    elements: list
    elem: np.ndarray
    mass: np.ndarray
    rtype: np.ndarray
    reac: np.ndarray
    prod: np.ndarray
    arr: np.ndarray
    troe: np.ndarray
    form: np.ndarray
    nasa: np.ndarray
    prow: np.ndarray
    lam: np.ndarray
    dlam: np.ndarray
    J0: np.ndarray
    sigma: np.ndarray
    sigma_abs: np.ndarray
    mu: float
    tf: float
    P_bar: np.ndarray
    T: np.ndarray
    Kzz: np.ndarray
    dcoef: np.ndarray
    g: float
    mbar: float
    alpha_T: float
    f0: np.ndarray
    # extinction by Rayleigh scattering and the diffuse field (Sec. 2.3.3), off unless given:
    # sigma_s[S, W] scattering cross sections (cm^2), albedo of the lower boundary, diffuse 1/0
    sigma_s: np.ndarray = None
    albedo: float = 0.0
    diffuse: int = 0

    @property
    def S(self):
        return int(self.elem.shape[0])

    @property
    def E(self):
        return int(self.elem.shape[1])

    @property
    def R(self):
        return int(self.rtype.shape[0])

    @property
    def L(self):
        return int(self.T.shape[0])

    @property
    def W(self):
        return int(self.lam.shape[0])

    @property
    def Rph(self):
        return int(self.sigma.shape[0])

    def replace(self, **kw):
        return dataclasses.replace(self, **kw)


# ---------------------------------------------------------------------------
# species
# ---------------------------------------------------------------------------

def _make_species(rng, elements, S):
    """Element-count vectors: H2 (bath), He (inert), the atoms, then random
    small molecules with 1-3 heavy atoms and 0-4 hydrogens, all distinct."""
    E = len(elements)
    idx = {e: i for i, e in enumerate(elements)}
    vecs = []
    seen = set()

    def add(v):
        t = tuple(int(x) for x in v)
        if t in seen or sum(t) == 0:
            return False
        seen.add(t)
        vecs.append(np.array(t, dtype=np.int32))
        return True

    v = np.zeros(E, np.int32); v[idx["H"]] = 2; add(v)          # H2, bath gas
    v = np.zeros(E, np.int32); v[idx["He"]] = 1; add(v)         # He, inert
    for e in elements:
        if e == "He":
            continue
        v = np.zeros(E, np.int32); v[idx[e]] = 1; add(v)        # atoms
    heavy = [e for e in elements if e not in ("H", "He")]
    # common elements are drawn more often, like real networks
    wt = np.array([{"C": 4, "O": 4, "N": 3, "S": 2}.get(e, 1.0) for e in heavy], float)
    wt /= wt.sum()
    tries = 0
    while len(vecs) < S:
        tries += 1
        if tries > 200000:
            raise RuntimeError("could not draw enough distinct species")
        nh = rng.choice([1, 2, 3], p=[0.45, 0.4, 0.15])
        v = np.zeros(E, np.int32)
        for e in rng.choice(len(heavy), size=nh, p=wt):
            v[idx[heavy[e]]] += 1
        v[idx["H"]] += rng.integers(0, 5)
        add(v)
    return np.stack(vecs[:S])


def _nasa_coeffs(rng, elem, elements):
    """Synthetic NASA-7 sets shaped like real molecules (Appendix A form).

    Per molecule with a atoms: C_p/R near 2.5 + 1.1 (a - 1) with small
    temperature terms; the enthalpy constant a6 holds a per-element part, a
    bond part of -4.2e4 K per bond (a - 1 bonds) and a random part eps_y; the
    entropy constant a7 gives S/R(1000 K) near 18 + 2 (a - 1).  Element parts
    cancel in any element-balanced reaction, so Gibbs energies of reaction are
    those of real chemistry in size.  Low and high sets are identical, so the
    polynomials are continuous at T_mid = 1000 K.  Returns (nasa, eps)."""
    S, E = elem.shape
    atoms = elem.sum(axis=1).astype(float)
    h_elem = rng.uniform(-2.0e4, 2.0e4, size=E)
    s_elem = rng.uniform(-1.0, 1.0, size=E)
    eps = rng.uniform(-8000.0, 8000.0, size=S)
    a1 = 2.5 + 1.1 * (atoms - 1.0) + rng.uniform(-0.3, 0.3, size=S)
    a2 = rng.uniform(-1e-3, 1e-3, size=S)
    a3 = rng.uniform(-1e-6, 1e-6, size=S)
    a4 = rng.uniform(-1e-9, 1e-9, size=S) * 0.3
    a5 = rng.uniform(-1e-13, 1e-13, size=S) * 0.3
    a6 = elem @ h_elem - 4.2e4 * (atoms - 1.0) + eps
    s_target = 18.0 + 2.0 * (atoms - 1.0) + elem @ s_elem + rng.uniform(-1.0, 1.0, size=S)
    a7 = s_target - a1 * np.log(1000.0)
    nasa = np.zeros((S, 15))
    nasa[:, 0] = 1000.0
    for base in (1, 8):
        nasa[:, base + 0] = a1
        nasa[:, base + 1] = a2
        nasa[:, base + 2] = a3
        nasa[:, base + 3] = a4
        nasa[:, base + 4] = a5
        nasa[:, base + 5] = a6
        nasa[:, base + 6] = a7
    # bath gas and inert He: plain monatomic/diatomic-like sets, eps = 0
    return nasa, eps


# ---------------------------------------------------------------------------
# reactions
# ---------------------------------------------------------------------------

def _pair_tables(elem, reactive):
    """Maps from the element vector of a pair sum to the unordered species
    pairs (i <= j) that have it, and from species vector to species index."""
    sums = {}
    ids = np.flatnonzero(reactive)
    for a_i, i in enumerate(ids):
        for j in ids[a_i:]:
            key = tuple((elem[i] + elem[j]).tolist())
            sums.setdefault(key, []).append((int(i), int(j)))
    single = {tuple(elem[i].tolist()): int(i) for i in ids}
    return sums, single


def _sample_arrhenius(rng, lo_exp, hi_exp, Tlo, Thi, kmax):
    """alpha log-uniform in [10^lo_exp, 10^hi_exp], beta U[-2,2], gamma U[0,3e4] K,
    Kooij form.  Draws are kept only if alpha (T/300)^beta stays below the
    collisional bound kmax at both ends of the profile's temperature range
    (the rate-validity criterion of Sec. 2.2)."""
    while True:
        alpha = 10.0 ** rng.uniform(lo_exp, hi_exp)
        beta = rng.uniform(-2.0, 2.0)
        gamma = rng.uniform(0.0, 3.0e4)
        top = alpha * max((Tlo / 300.0) ** beta, (Thi / 300.0) ** beta)
        if top <= kmax:
            return alpha, beta, gamma


def _make_reactions(rng, elem, eps, n_two, n_three, n_photo, Tlo, Thi):
    S = elem.shape[0]
    reactive = np.ones(S, bool)
    reactive[1] = False                    # He takes no part in chemistry
    sums, single = _pair_tables(elem, reactive)
    groups = [v for v in sums.values() if len(v) >= 2]
    if n_two and not groups:
        raise RuntimeError("no balanced two-body reactions possible")

    rtype, reac, prod, arr, troe, form = [], [], [], [], [], []
    seen = set()

    def push(t, r, p, a, tr, f):
        rtype.append(t); reac.append(r + [-1] * (3 - len(r))); prod.append(p + [-1] * (3 - len(p)))
        arr.append(a); troe.append(tr); form.append(f)

    # two-body A + B <-> C + D, oriented so that the random enthalpy part
    # sum(nu * eps) is not positive (the exothermic direction is the forward one)
    guard = 0
    while sum(1 for t in rtype if t == RX_TWO_BODY) < n_two:
        guard += 1
        if guard > 50 * n_two + 10000:
            raise RuntimeError("could not draw enough two-body reactions")
        g = groups[rng.integers(len(groups))]
        a, b = rng.choice(len(g), size=2, replace=False)
        p1, p2 = g[a], g[b]
        key = (min(p1, p2), max(p1, p2))
        if key in seen:
            continue
        seen.add(key)
        d = eps[p2[0]] + eps[p2[1]] - eps[p1[0]] - eps[p1[1]]
        if d > 0:
            p1, p2 = p2, p1
        al, be, ga = _sample_arrhenius(rng, -14.0, -9.0, Tlo, Thi, 1e-9)
        push(RX_TWO_BODY, list(p1), list(p2), [al, be, ga] + [0.0] * 6, [0.0] * 4, FORM_KOOIJ)

    # three-body association A + B (+M) <-> C with Troe fall-off
    assoc = []
    for key, pairs in sums.items():
        c = single.get(key)
        if c is None:
            continue
        for pr in pairs:
            if c not in pr:
                assoc.append((pr, c))
    if n_three and not assoc:
        raise RuntimeError("no association reactions possible")
    order = rng.permutation(len(assoc))
    used = 0
    for oi in order:
        if used >= n_three:
            break
        pr, c = assoc[oi]
        key = ("3", pr, c)
        if key in seen:
            continue
        seen.add(key)
        a0, b0, g0 = _sample_arrhenius(rng, -36.0, -28.0, Tlo, Thi, 1e-28)
        ai, bi, gi = _sample_arrhenius(rng, -12.0, -9.0, Tlo, Thi, 1e-9)
        fc = rng.uniform(0.3, 0.9)
        push(RX_THREE_BODY, list(pr), [c], [0.0, 0.0, 0.0, a0, b0, g0, ai, bi, gi],
             [fc, 1e-30, 1e30, 0.0], FORM_KOOIJ)
        used += 1
    if used < n_three:
        # reuse association channels with fresh parameters if the species set is small
        while used < n_three:
            pr, c = assoc[rng.integers(len(assoc))]
            a0, b0, g0 = _sample_arrhenius(rng, -36.0, -28.0, Tlo, Thi, 1e-28)
            ai, bi, gi = _sample_arrhenius(rng, -12.0, -9.0, Tlo, Thi, 1e-9)
            fc = rng.uniform(0.3, 0.9)
            push(RX_THREE_BODY, list(pr), [c], [0.0, 0.0, 0.0, a0, b0, g0, ai, bi, gi],
                 [fc, 1e-30, 1e30, 0.0], FORM_KOOIJ)
            used += 1

    # photodissociation A -> B + C (irreversible)
    photo = [(c, pr) for (pr, c) in assoc]
    order = rng.permutation(len(photo)) if photo else []
    prow = []
    used = 0
    chosen = []
    for oi in order:
        if used >= n_photo:
            break
        c, pr = photo[oi]
        key = ("p", c, pr)
        if key in seen:
            continue
        seen.add(key)
        chosen.append((c, pr))
        used += 1
    if used < n_photo:
        raise RuntimeError("not enough photodissociation channels")
    for c, pr in chosen:
        push(RX_PHOTO, [c], list(pr), [0.0] * 9, [0.0] * 4, FORM_KOOIJ)

    R = len(rtype)
    prow = -np.ones(R, np.int32)
    ph = [i for i, t in enumerate(rtype) if t == RX_PHOTO]
    prow[ph] = np.arange(len(ph), dtype=np.int32)
    return (np.array(rtype, np.int32), np.array(reac, np.int32), np.array(prod, np.int32),
            np.array(arr, float), np.array(troe, float), np.array(form, np.int32), prow)


# ---------------------------------------------------------------------------
# photolysis inputs
# ---------------------------------------------------------------------------

_H = 6.62607015e-27     # erg s
_C = 2.99792458e10      # cm / s
_KB = 1.380649e-16      # erg / K
_RSUN = 6.957e10        # cm
_AU = 1.495978707e13    # cm


def _stellar_photon_flux(lam_A, Tstar=5000.0, rstar=0.8 * _RSUN, a=0.03 * _AU):
    """Black-body photon flux at the planet, photons cm^-2 s^-1 A^-1:
    pi B_lambda / (h c / lambda), scaled by (R*/a)^2 (the (r/a)^2 rescaling
    of stellar spectra described with the actinic flux)."""
    lam = lam_A * 1e-8
    x = _H * _C / (lam * _KB * Tstar)
    with np.errstate(over="ignore"):                               # far-UV bins of a cool star: B -> 0
        B = 2.0 * _H * _C ** 2 / lam ** 5 / np.expm1(x)          # erg s^-1 cm^-2 cm^-1 sr^-1
    photons = np.pi * B / (_H * _C / lam) * 1e-8                   # per Angstrom
    return photons * (rstar / a) ** 2


def _photo_inputs(rng, W, Rph, reac, prow, S):
    edges = np.geomspace(500.0, 5000.0, W + 1)
    lam = 0.5 * (edges[1:] + edges[:-1])
    dlam = np.diff(edges)
    J0 = _stellar_photon_flux(lam)
    sigma = np.zeros((Rph, W))
    for i in range(Rph):
        peak = 10.0 ** rng.uniform(-19.0, -16.0)
        centre = rng.uniform(1000.0, 2500.0)
        width = rng.uniform(0.1, 0.3)
        sigma[i] = peak * np.exp(-np.log(lam / centre) ** 2 / (2.0 * width ** 2))
    sigma_abs = np.zeros((S, W))
    for r in np.flatnonzero(prow >= 0):
        sigma_abs[reac[r, 0]] += sigma[prow[r]]     # absorption taken as the sum of dissociation channels
    return lam, dlam, J0, sigma, sigma_abs


def rayleigh_cross_sections(elem, elements, lam):
    """Rayleigh scattering cross sections sigma_s[S, W] (cm^2), lambda^-4 in shape: H2 at
    8.14e-13 / lambda^4 (lambda in Angstrom), He at 0.0838 times that, and every other species in
    proportion to the square of its atom count (polarisability grows with size) times H2's per atom
    pair; species are drawn as scatterers only if they hold at most three atoms."""
    S = elem.shape[0]
    atoms = elem.sum(axis=1).astype(float)
    base = 8.14e-13 / lam ** 4
    sig = np.zeros((S, lam.shape[0]))
    for y in range(S):
        if y == 0:
            sig[y] = base                                  # H2, the bath gas
        elif y == 1:
            sig[y] = 0.0838 * base                         # He
        elif atoms[y] <= 3:
            sig[y] = base * (atoms[y] / 2.0) ** 2
    return sig


def with_scattering(prob, albedo=0.0, diffuse=1, bins=None):
    """The same column with Rayleigh scattering in the extinction and the diffuse field on.  With
    bins, the photolysis grid becomes `bins` bins of about 1 A from 1 A to 10,000 A (the paper's
    10,000-bin grid at bins=10000), the cross sections redrawn on it with the same seeds."""
    if bins is not None:
        rng = np.random.default_rng(1234)
        edges = np.linspace(1.0, 10000.0, bins + 1)
        lam = 0.5 * (edges[1:] + edges[:-1])
        dlam = np.diff(edges)
        J0 = _stellar_photon_flux(lam)
        Rph = prob.Rph
        sigma = np.zeros((Rph, bins))
        for i in range(Rph):
            peak = 10.0 ** rng.uniform(-19.0, -16.0)
            centre = rng.uniform(1000.0, 2500.0)
            width = rng.uniform(0.1, 0.3)
            sigma[i] = peak * np.exp(-np.log(lam / centre) ** 2 / (2.0 * width ** 2))
        sigma_abs = np.zeros((prob.S, bins))
        for r in np.flatnonzero(prob.prow >= 0):
            sigma_abs[prob.reac[r, 0]] += sigma[prob.prow[r]]
        prob = prob.replace(lam=lam, dlam=dlam, J0=J0, sigma=sigma, sigma_abs=sigma_abs)
    sig_s = rayleigh_cross_sections(prob.elem, prob.elements, prob.lam)
    return prob.replace(sigma_s=sig_s, albedo=float(albedo), diffuse=int(diffuse),
                        name=prob.name + f"-rt{prob.W}")


# ---------------------------------------------------------------------------
# atmosphere profiles
# ---------------------------------------------------------------------------

def profile_tiny(L=40):
    P = np.geomspace(1e2, 1e-6, L)
    T = 1500.0 + (1000.0 - 1500.0) * (np.log10(1e2) - np.log10(P)) / (np.log10(1e2) - np.log10(1e-6))
    Kzz = np.full(L, 1e8)
    return P, T, Kzz


def profile_hot_jupiter(L=150, T_scale=1.0, Kzz_scale=1.0):
    """150 layers 1e2 -> 1e-8 bar; T = 1000 + 800 (1 + tanh(log10 P + 1)) / 2 K
    (about 1,800 K deep, 1,000 K at the top); Kzz = 1e7 (P / 100 bar)^-0.5
    clipped at 1e10 cm^2/s."""
    P = np.geomspace(1e2, 1e-8, L)
    T = (1000.0 + 800.0 * 0.5 * (1.0 + np.tanh(np.log10(P) + 1.0))) * T_scale
    Kzz = np.minimum(1e7 * (P / 1e2) ** -0.5, 1e10) * Kzz_scale
    return P, T, Kzz


def _initial_mixing(rng, elem, L, metallicity=1.0):
    """User-defined initial composition: H2 0.85, trace species at
    10^U[-10,-5] times metallicity, He the remainder, floored at 1e-30;
    the same at every layer."""
    S = elem.shape[0]
    f = 10.0 ** rng.uniform(-10.0, -5.0, size=S) * metallicity
    f[0] = 0.85
    f[1] = 0.0
    f[1] = max(0.15 - f[2:].sum(), 1e-3)
    f = np.maximum(f, 1e-30)
    return np.tile(f, (L, 1))


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

CONFIG_ELEMENTS = {
    "cho": ["H", "He", "C", "O"],
    "chons": ["H", "He", "C", "O", "N", "S"],
    "full": ["H", "He", "C", "O", "N", "P", "S", "Na", "K", "Fe", "Mg", "Si", "Ti", "Cl"],
}


def make_problem(name, S, n_two, n_three, n_photo, elements, profile, seed,
                 W=1000, D0=1.0e17, metallicity=1.0, mu=0.5, tf=0.5):
    rng = np.random.default_rng(seed)
    P, T, Kzz = profile
    L = P.shape[0]
    elem = _make_species(rng, elements, S)
    masses = np.array([ELEMENT_MASS[e] for e in elements])
    mass = elem @ masses
    nasa, eps = _nasa_coeffs(rng, elem, elements)
    Tlo, Thi = float(T.min()), float(T.max())
    rtype, reac, prod, arr, troe, form, prow = _make_reactions(
        rng, elem, eps, n_two, n_three, n_photo, Tlo, Thi)
    Rph = int((prow >= 0).sum())
    if Rph:
        lam, dlam, J0, sigma, sigma_abs = _photo_inputs(rng, W, Rph, reac, prow, S)
    else:
        lam = np.zeros(0); dlam = np.zeros(0); J0 = np.zeros(0)
        sigma = np.zeros((0, 0)); sigma_abs = np.zeros((S, 0))
    m_bath = 2.016
    dcoef = D0 * np.sqrt(1.0 / mass + 1.0 / m_bath)
    f0 = _initial_mixing(rng, elem, L, metallicity)
    return Problem(name=name, elements=list(elements), elem=elem.astype(np.int32), mass=mass,
                   rtype=rtype, reac=reac, prod=prod, arr=arr, troe=troe, form=form,
                   nasa=nasa, prow=prow, lam=lam, dlam=dlam, J0=J0, sigma=sigma,
                   sigma_abs=sigma_abs, mu=mu, tf=tf, P_bar=P.astype(float), T=T.astype(float),
                   Kzz=Kzz.astype(float), dcoef=dcoef, g=2.0e3, mbar=2.3, alpha_T=0.0, f0=f0)


def tiny_column(seed=0):
    """20 species over C/H/O, 60 element-balanced A+B->C+D reactions, 40
    layers 1e2 -> 1e-6 bar, T 1500 -> 1000 K, Kzz = 1e8, no photolysis."""
    return make_problem("tiny-20sp-60rx-40L", 20, 60, 0, 0, CONFIG_ELEMENTS["cho"],
                        profile_tiny(40), seed)


def chons_column(seed=1, L=150):
    """96 species over C/H/O/N/S, 1,200 thermal reactions (20 % three-body with
    Troe fall-off) plus 40 photodissociations, 1,000 wavelength bins, 150 layers."""
    return make_problem("chons-96sp-1240rx-150L", 96, 960, 240, 40, CONFIG_ELEMENTS["chons"],
                        profile_hot_jupiter(L), seed)


def full_column(seed=2, L=150):
    """594 species over C-H-O-N-P-S plus metals, 7,720 reactions (7,520
    thermal, 20 % three-body, plus 200 photodissociations), 150 layers."""
    return make_problem("xodiac-594sp-7720rx-150L", 594, 6016, 1504, 200, CONFIG_ELEMENTS["full"],
                        profile_hot_jupiter(L), seed)


def small_column(S=40, L=60, n_two=120, n_three=30, n_photo=10, seed=5, W=200, elements="chons"):
    """Mid-size test column: several tiles in each dimension with ragged tails."""
    elems = CONFIG_ELEMENTS[elements]
    return make_problem(f"small-{S}sp-{L}L", S, n_two, n_three, n_photo, elems,
                        profile_hot_jupiter(L), seed, W=W)


def sweep_column(S, L, T_eq, metallicity, kzz_scale, seed):
    """One column of a planet-parameter sweep: the hot-Jupiter profile scaled
    by T_eq / 1400 K, the Kzz profile scaled, trace abundances scaled by the
    metallicity."""
    sizes = {96: (960, 240, 40, "chons"), 250: (2600, 650, 80, "full"), 594: (6016, 1504, 200, "full")}
    n_two, n_three, n_ph, el = sizes[S]
    return make_problem(f"sweep-{S}sp-{L}L", S, n_two, n_three, n_ph, CONFIG_ELEMENTS[el],
                        profile_hot_jupiter(L, T_scale=T_eq / 1400.0, Kzz_scale=kzz_scale),
                        seed, metallicity=metallicity)
