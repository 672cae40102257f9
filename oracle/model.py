"""Lattice, couplings and the product-term list of Eq. (1) + Eq. (16).
Test infrastructure only.

Every Hamiltonian term is written as a coefficient times a product of
genuinely local (fermion-even) site operators, so sites can be treated as
plain tensor factors (Methods: the factorisations of Eq. (15) and of the
plaquette make every operator local and bosonic).

Readings of the paper used here (the library takes the same ones):
* couplings t, m, ge2 = g_e^2, cB, nu are independent inputs; the plaquette
  enters as -cB * sum(box + h.c.) (Eq. (1) third line with cB = g_m^2/2);
* open boundaries keep all six half-links at every site; half-links that
  point out of the lattice are "dangling": no hopping, plaquette or penalty
  acts on them and each costs (ge2/2)(1 - k)^2;
* the electric energy of an internal link (x, +mu) is (ge2/2)(1 - k_{x,+mu})^2
  read on the lower site, Eq. (10);
* the penalty of Eq. (16), nu * (1 - delta_{2,L}) per internal link, is
  written as nu * sum_k P^k_{x,+mu} (x) (1 - P^{2-k}_{x+mu,-mu}) (exact,
  since sum_k P^k = 1), so no additive constant remains;
* periodic boundaries (Results, "Transition at zero charge"): every
  direction with more than one site wraps around (an extent of 2 gives two
  links between the same two sites); a direction of extent 1 stays open;
* local chemical potentials (Methods: diagonal local terms that pin
  charges; Results, "Quantum capacitor"): mu_x psi^dag_x psi_x per site, a
  class of its own ('mu').
"""
from dataclasses import dataclass, field, replace

# half-link index (0-based): -x, -y, -z, +x, +y, +z
def minus(mu):
    return mu


def plus(mu):
    return 3 + mu


@dataclass(frozen=True)
class Params:
    """Couplings and lattice of Eq. (1) + Eq. (16).  ``Q`` is the total
    charge sum_x (phi_x - (1 - p_x)/2)."""
    Lx: int
    Ly: int
    Lz: int
    t: float = 1.0
    m: float = 1.0
    ge2: float = 1.0
    cB: float = 0.5
    nu: float = 10.0
    Q: int = 0
    boundary: int = 0          # 0 open, 1 periodic
    mu: tuple = ()             # chemical potential per site (empty: none)


@dataclass(frozen=True)
class Term:
    """coef * prod_{(site, key) in ops} O_key(site).  ``cls`` names the
    coupling the coefficient is proportional to ('t', 'm', 'ge2', 'cB',
    'nu'); ``unit`` = coef / coupling."""
    coef: float
    cls: str
    unit: float
    ops: tuple


@dataclass
class Lattice:
    Lx: int
    Ly: int
    Lz: int
    periodic: bool = False

    @property
    def n_sites(self):
        return self.Lx * self.Ly * self.Lz

    def index(self, i, j, k):
        return i + self.Lx * (j + self.Ly * k)

    def coords(self, s):
        i = s % self.Lx
        j = (s // self.Lx) % self.Ly
        k = s // (self.Lx * self.Ly)
        return (i, j, k)

    def dims(self):
        return (self.Lx, self.Ly, self.Lz)

    def inside(self, c):
        return all(0 <= c[a] < self.dims()[a] for a in range(3))

    def parity(self, s):
        """(-1)^(i+j+k); site (0,0,0) is even (Eq. (1) text)."""
        return 1 if sum(self.coords(s)) % 2 == 0 else -1

    def neighbour(self, s, mu, step=1):
        c = list(self.coords(s))
        c[mu] += step
        if self.periodic and self.dims()[mu] > 1:
            c[mu] %= self.dims()[mu]
        return self.index(*c) if self.inside(c) else None

    def links(self):
        """Internal links (x, mu, y = x + mu) in site order, then mu."""
        out = []
        for s in range(self.n_sites):
            for mu in range(3):
                y = self.neighbour(s, mu)
                if y is not None:
                    out.append((s, mu, y))
        return out

    def plaquettes(self):
        """(x, mu, nu) with mu < nu and all four corners inside."""
        out = []
        for s in range(self.n_sites):
            for mu in range(3):
                for nu in range(mu + 1, 3):
                    a = self.neighbour(s, mu)
                    b = self.neighbour(s, nu)
                    if a is None or b is None:
                        continue
                    c = self.neighbour(a, nu)
                    out.append((s, mu, nu, a, c, b))
        return out

    def dangling(self, s):
        """Half-links of site s that point out of the lattice."""
        out = []
        for mu in range(3):
            if self.neighbour(s, mu, -1) is None:
                out.append(minus(mu))
            if self.neighbour(s, mu, +1) is None:
                out.append(plus(mu))
        return tuple(sorted(out))

    def electric_mask(self, s):
        """Half-links whose E^2 is charged to site s: its internal +mu
        half-links and its dangling ones."""
        mask = set(self.dangling(s))
        for mu in range(3):
            if self.neighbour(s, mu, +1) is not None:
                mask.add(plus(mu))
        return tuple(sorted(mask))


def lattice(p: Params):
    """The lattice of p (open or periodic)."""
    return Lattice(p.Lx, p.Ly, p.Lz, periodic=(p.boundary == 1))


def build_terms(p: Params):
    """Product terms of Eq. (1) + Eq. (16) and the constant nu * N_links.

    Returns (terms, constant).  Site ops are keys understood by
    ``oracle.fock.site_op``."""
    lat = lattice(p)
    terms = []
    # staggered mass m sum_x (-1)^x psi^dag psi  (Eq. (1), second line)
    for s in range(lat.n_sites):
        par = lat.parity(s)
        terms.append(Term(p.m * par, "m", float(par), ((s, ("n",)),)))
    # electric energy ge2/2 sum E^2 (Eq. (1) second line, Eq. (10))
    for s in range(lat.n_sites):
        mask = lat.electric_mask(s)
        if mask:
            terms.append(Term(0.5 * p.ge2, "ge2", 0.5, ((s, ("E2", mask)),)))
    # hopping -t (psi_x^dag U psi_y + h.c.) = -t (M_x M'_y + M'^dag...), Eq. (15)
    for (x, mu, y) in lat.links():
        terms.append(Term(-p.t, "t", -1.0, ((x, ("M", plus(mu))), (y, ("Md", minus(mu))))))
        terms.append(Term(-p.t, "t", -1.0, ((x, ("Md", plus(mu))), (y, ("M", minus(mu))))))
    # plaquette -cB (box + h.c.) with box = -C_x C_{x+mu} C_{x+mu+nu} C_{x+nu}
    for (x, mu, nu, a, c, b) in lat.plaquettes():
        fwd = (
            (x, ("C", plus(nu), plus(mu))),
            (a, ("C", minus(mu), plus(nu))),
            (c, ("C", minus(nu), minus(mu))),
            (b, ("C", plus(mu), minus(nu))),
        )
        bwd = tuple((s, ("C", key[2], key[1])) for (s, key) in fwd)
        terms.append(Term(p.cB, "cB", 1.0, tuple(sorted(fwd))))
        terms.append(Term(p.cB, "cB", 1.0, tuple(sorted(bwd))))
    # penalty nu sum (1 - delta_{2,L}), Eq. (16), written with sum_k P^k = 1 as
    # nu sum_k P^k_{x,+mu} (1 - P^{2-k}_{y,-mu}): three non-negative product
    # terms per link and no additive constant
    links = lat.links()
    for (x, mu, y) in links:
        for k in range(3):
            terms.append(Term(p.nu, "nu", 1.0, ((x, ("P", plus(mu), k)), (y, ("PC", minus(mu), 2 - k)))))
    # local chemical potentials mu_x psi^dag_x psi_x
    for s, mu_s in enumerate(p.mu):
        terms.append(Term(float(mu_s), "mu", 1.0, ((s, ("n",)),)))
    constant = 0.0
    # drop exactly-zero couplings: they contribute nothing
    terms = [tm for tm in terms if tm.coef != 0.0]
    return terms, constant


def with_couplings(p: Params, **kw):
    return replace(p, **kw)


def class_only(p: Params, cls):
    """Params keeping only the coupling ``cls`` (others set to zero)."""
    zero = dict(t=0.0, m=0.0, ge2=0.0, cB=0.0, nu=0.0, mu=())
    zero[cls] = getattr(p, cls)
    return replace(p, **zero)
