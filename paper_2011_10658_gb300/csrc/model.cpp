// Host model: dressed-site basis (Eq. (12)-(14)), monomial site operators
// from the closed-form Jordan-Wigner sign of the rishon modes (Eq. (6)),
// product terms of Eq. (1) + Eq. (16), binary tree and U(1) sectors.
#include "model.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <stdexcept>

namespace qed {

// ---------------------------------------------------------------- basis
// Rows: phi outer (0, 1), then (k1..k6) lexicographic, k1 most significant;
// kept iff phi + sum k = 6 + (1 - p)/2 (Eq. (14)).  Sign of Eq. (12):
// (-1)^{[k1=2]+[k2=2]+[k3=2]}.  Charge q = phi - (1 - p)/2.
void enumerate_basis(int parity, int8_t* table) {
  const int target = 6 + (1 - parity) / 2;
  int n = 0;
  for (int phi = 0; phi < 2; ++phi) {
    for (int code = 0; code < 729; ++code) {
      int k[6];
      int c = code;
      for (int j = 5; j >= 0; --j) { k[j] = c % 3; c /= 3; }
      int sum = phi;
      for (int j = 0; j < 6; ++j) sum += k[j];
      if (sum != target) continue;
      int8_t* row = table + 9 * n;
      row[0] = (int8_t)phi;
      for (int j = 0; j < 6; ++j) row[1 + j] = (int8_t)k[j];
      int twos = (k[0] == 2) + (k[1] == 2) + (k[2] == 2);
      row[7] = (int8_t)((twos & 1) ? -1 : 1);
      row[8] = (int8_t)(phi - (1 - parity) / 2);
      ++n;
    }
  }
  if (n != kLocalDim) throw std::logic_error("dressed basis size");
}

namespace {

struct BasisCache {
  int8_t table[2][kLocalDim * 9];
  std::map<uint32_t, int> index[2];   // packed (phi, k) -> row
  BasisCache() {
    for (int t = 0; t < 2; ++t) {
      int parity = t == 0 ? 1 : -1;
      enumerate_basis(parity, table[t]);
      for (int r = 0; r < kLocalDim; ++r) index[t][pack(table[t] + 9 * r)] = r;
    }
  }
  static uint32_t pack(const int8_t* row) {
    uint32_t v = (uint32_t)row[0];
    for (int j = 0; j < 6; ++j) v = v * 3 + (uint32_t)row[1 + j];
    return v;
  }
};

const BasisCache& basis_cache() {
  static BasisCache c;
  return c;
}

// Occupation state of one site in the Fock representation used to derive
// the signs: phi and the six half-link occupations.
struct FockState {
  int phi;
  int k[6];
  int coef;   // accumulated +-1, 0 = annihilated
};

// eta_j^dag: k_j -> k_j + 1 (zero at k_j = 2), sign (-1)^{phi + sum_{i<j} k_i}:
// eta^dag is fermion-odd and must pass psi^dag and the creation strings of
// half-links 1..j-1 (each of length k_i) in (psi^dag)^phi c_1 ... c_6 |0>.
// Within the half-link, Eq. (6) maps |0> -> a^dag|0> and a^dag|0> ->
// b^dag a^dag|0> with amplitude +1.
void apply_eta_dag(FockState* s, int j) {
  if (s->coef == 0) return;
  if (s->k[j] == 2) { s->coef = 0; return; }
  int pre = s->phi;
  for (int i = 0; i < j; ++i) pre += s->k[i];
  if (pre & 1) s->coef = -s->coef;
  s->k[j] += 1;
}

// eta_j: the adjoint, k_j -> k_j - 1 with the same prefix sign.
void apply_eta(FockState* s, int j) {
  if (s->coef == 0) return;
  if (s->k[j] == 0) { s->coef = 0; return; }
  int pre = s->phi;
  for (int i = 0; i < j; ++i) pre += s->k[i];
  if (pre & 1) s->coef = -s->coef;
  s->k[j] -= 1;
}

// psi is the first mode: no sign.
void apply_psi_dag(FockState* s) {
  if (s->coef == 0) return;
  if (s->phi == 1) { s->coef = 0; return; }
  s->phi = 1;
}

void apply_psi(FockState* s) {
  if (s->coef == 0) return;
  if (s->phi == 0) { s->coef = 0; return; }
  s->phi = 0;
}

}  // namespace

int site_charge(int parity, int row) {
  return basis_cache().table[parity == 1 ? 0 : 1][9 * row + 8];
}

void build_site_op(int parity, const OpKey& key, SiteOp* out) {
  const BasisCache& bc = basis_cache();
  const int t = parity == 1 ? 0 : 1;
  const int8_t* tab = bc.table[t];
  for (int r = 0; r < kLocalDim; ++r) { out->src[r] = -1; out->val[r] = 0.0; }
  out->dq = 0;
  if (key.kind == OP_M) out->dq = 1;
  if (key.kind == OP_MD) out->dq = -1;
  for (int in = 0; in < kLocalDim; ++in) {
    const int8_t* row = tab + 9 * in;
    if (key.kind == OP_IDENTITY) { out->src[in] = (int16_t)in; out->val[in] = 1.0; continue; }
    if (key.kind == OP_P) {
      if (row[1 + key.a] == key.b) { out->src[in] = (int16_t)in; out->val[in] = 1.0; }
      continue;
    }
    if (key.kind == OP_PC) {
      if (row[1 + key.a] != key.b) { out->src[in] = (int16_t)in; out->val[in] = 1.0; }
      continue;
    }
    if (key.kind == OP_N) {
      if (row[0] == 1) { out->src[in] = (int16_t)in; out->val[in] = 1.0; }
      continue;
    }
    if (key.kind == OP_E2) {
      double v = 0.0;
      for (int j = 0; j < 6; ++j)
        if (key.a & (1 << j)) { double e = 1.0 - row[1 + j]; v += e * e; }
      if (v != 0.0) { out->src[in] = (int16_t)in; out->val[in] = v; }
      continue;
    }
    FockState s;
    s.phi = row[0];
    for (int j = 0; j < 6; ++j) s.k[j] = row[1 + j];
    s.coef = 1;
    // operators act right to left on the input state
    if (key.kind == OP_M) { apply_eta(&s, key.a); apply_psi_dag(&s); }
    else if (key.kind == OP_MD) { apply_psi(&s); apply_eta_dag(&s, key.a); }
    else if (key.kind == OP_C) { apply_eta(&s, key.b); apply_eta_dag(&s, key.a); }
    else throw std::invalid_argument("site op kind");
    if (s.coef == 0) continue;
    int8_t packed[9];
    packed[0] = (int8_t)s.phi;
    for (int j = 0; j < 6; ++j) packed[1 + j] = (int8_t)s.k[j];
    auto it = bc.index[t].find(BasisCache::pack(packed));
    if (it == bc.index[t].end()) throw std::logic_error("operator leaves the gauge-invariant basis");
    const int outr = it->second;
    // dressed rows carry the Eq. (12) sign on both sides
    const int sign = s.coef * tab[9 * outr + 7] * row[7];
    out->src[outr] = (int16_t)in;
    out->val[outr] = (double)sign;
  }
}

// ---------------------------------------------------------------- lattice
void Lattice::coords(int s, int c[3]) const {
  c[0] = s % Lx;
  c[1] = (s / Lx) % Ly;
  c[2] = s / (Lx * Ly);
}

int Lattice::parity(int s) const {
  int c[3];
  coords(s, c);
  return ((c[0] + c[1] + c[2]) % 2 == 0) ? 1 : -1;
}

int Lattice::neighbour(int s, int mu, int step) const {
  int c[3];
  coords(s, c);
  c[mu] += step;
  const int dims[3] = {Lx, Ly, Lz};
  if (periodic && dims[mu] > 1) c[mu] = ((c[mu] % dims[mu]) + dims[mu]) % dims[mu];
  if (c[mu] < 0 || c[mu] >= dims[mu]) return -1;
  return index(c[0], c[1], c[2]);
}

std::vector<int> Lattice::dangling(int s) const {
  std::vector<int> out;
  for (int mu = 0; mu < 3; ++mu) {
    if (neighbour(s, mu, -1) < 0) out.push_back(mu);
    if (neighbour(s, mu, +1) < 0) out.push_back(3 + mu);
  }
  std::sort(out.begin(), out.end());
  return out;
}

int Lattice::electric_mask(int s) const {
  int mask = 0;
  for (int j : dangling(s)) mask |= 1 << j;
  for (int mu = 0; mu < 3; ++mu)
    if (neighbour(s, mu, +1) >= 0) mask |= 1 << (3 + mu);
  return mask;
}

int Lattice::n_links() const {
  int n = 0;
  for (int s = 0; s < n_sites(); ++s)
    for (int mu = 0; mu < 3; ++mu) n += neighbour(s, mu, +1) >= 0;
  return n;
}

static OpKey key(int kind, int a = 0, int b = 0) {
  OpKey k;
  k.kind = kind;
  k.a = a;
  k.b = b;
  return k;
}

// Eq. (1) + Eq. (16) as coefficient x product of local ops.  Same order as
// the terms are listed: mass, electric, hopping, plaquette, penalty.
void build_terms(const Params& p, std::vector<Term>* terms, double* constant) {
  Lattice lat{p.Lx, p.Ly, p.Lz, p.boundary == 1};
  terms->clear();
  const int n = lat.n_sites();
  auto push = [&](double coef, int cls, std::vector<std::pair<int, OpKey>> ops) {
    if (coef == 0.0) return;
    std::sort(ops.begin(), ops.end(), [](const std::pair<int, OpKey>& x, const std::pair<int, OpKey>& y) {
      return x.first < y.first;
    });
    Term t;
    t.coef = coef;
    t.cls = cls;
    t.ops = std::move(ops);
    terms->push_back(std::move(t));
  };
  for (int s = 0; s < n; ++s) push(p.m * lat.parity(s), CLS_M, {{s, key(OP_N)}});
  for (int s = 0; s < n; ++s) {
    int mask = lat.electric_mask(s);
    if (mask) push(0.5 * p.ge2, CLS_GE2, {{s, key(OP_E2, mask)}});
  }
  int n_links = 0;
  for (int x = 0; x < n; ++x)
    for (int mu = 0; mu < 3; ++mu) {
      int y = lat.neighbour(x, mu, +1);
      if (y < 0) continue;
      ++n_links;
      push(-p.t, CLS_T, {{x, key(OP_M, 3 + mu)}, {y, key(OP_MD, mu)}});
      push(-p.t, CLS_T, {{x, key(OP_MD, 3 + mu)}, {y, key(OP_M, mu)}});
    }
  for (int x = 0; x < n; ++x)
    for (int mu = 0; mu < 3; ++mu)
      for (int nu = mu + 1; nu < 3; ++nu) {
        int a = lat.neighbour(x, mu, +1);
        int b = lat.neighbour(x, nu, +1);
        if (a < 0 || b < 0) continue;
        int c = lat.neighbour(a, nu, +1);
        // box = -C_x C_{x+mu} C_{x+mu+nu} C_{x+nu}; -cB (box + h.c.) = +cB (CCCC + h.c.)
        std::vector<std::pair<int, OpKey>> fwd = {{x, key(OP_C, 3 + nu, 3 + mu)},
                                                  {a, key(OP_C, mu, 3 + nu)},
                                                  {c, key(OP_C, nu, mu)},
                                                  {b, key(OP_C, 3 + mu, nu)}};
        std::vector<std::pair<int, OpKey>> bwd;
        for (auto& f : fwd) bwd.push_back({f.first, key(OP_C, f.second.b, f.second.a)});
        push(p.cB, CLS_CB, fwd);
        push(p.cB, CLS_CB, bwd);
      }
  for (int x = 0; x < n; ++x)
    for (int mu = 0; mu < 3; ++mu) {
      int y = lat.neighbour(x, mu, +1);
      if (y < 0) continue;
      // nu (1 - delta_{2,L}) = nu sum_k P^k_x (1 - P^{2-k}_y): non-negative terms, no constant
      for (int k = 0; k < 3; ++k) push(p.nu, CLS_NU, {{x, key(OP_P, 3 + mu, k)}, {y, key(OP_PC, mu, 2 - k)}});
    }
  (void)n_links;
  // local chemical potentials mu_x psi^dag_x psi_x (diagonal, own class)
  for (int s = 0; s < n && s < (int)p.mu.size(); ++s) push(p.mu[s], CLS_MU, {{s, key(OP_N)}});
  *constant = 0.0;
}

// ---------------------------------------------------------------- tree
std::vector<TreeNode> build_tree(int Lx, int Ly, int Lz) {
  Lattice lat{Lx, Ly, Lz};
  const int dims[3] = {Lx, Ly, Lz};
  struct Block { int kind, id; int lo[3], hi[3]; std::vector<int> sites; };
  std::vector<Block> blocks;
  for (int s = 0; s < lat.n_sites(); ++s) {
    Block b;
    b.kind = 0;
    b.id = s;
    int c[3];
    lat.coords(s, c);
    for (int a = 0; a < 3; ++a) { b.lo[a] = c[a]; b.hi[a] = c[a] + 1; }
    b.sites = {s};
    blocks.push_back(b);
  }
  std::vector<TreeNode> nodes;
  int layer = 0, axis = 0;
  while (blocks.size() > 1) {
    for (int tries = 0; tries < 3; ++tries) {
      int ext = blocks[0].hi[axis] - blocks[0].lo[axis];
      if (ext < dims[axis]) break;
      axis = (axis + 1) % 3;
    }
    const int ext = blocks[0].hi[axis] - blocks[0].lo[axis];
    struct Merge { int lo[3], hi[3]; int left, right; };
    std::vector<Merge> merges;
    for (size_t i = 0; i < blocks.size(); ++i) {
      const Block& b = blocks[i];
      if ((b.lo[axis] / ext) % 2 != 0) continue;
      int want[3] = {b.lo[0], b.lo[1], b.lo[2]};
      want[axis] += ext;
      int partner = -1;
      for (size_t j = 0; j < blocks.size(); ++j)
        if (blocks[j].lo[0] == want[0] && blocks[j].lo[1] == want[1] && blocks[j].lo[2] == want[2]) partner = (int)j;
      if (partner < 0) throw std::logic_error("tree: lattice extents must be powers of two");
      Merge m;
      for (int a = 0; a < 3; ++a) { m.lo[a] = b.lo[a]; m.hi[a] = b.hi[a]; }
      m.hi[axis] = blocks[partner].hi[axis];
      m.left = (int)i;
      m.right = partner;
      merges.push_back(m);
    }
    std::sort(merges.begin(), merges.end(), [](const Merge& x, const Merge& y) {
      if (x.lo[2] != y.lo[2]) return x.lo[2] < y.lo[2];
      if (x.lo[1] != y.lo[1]) return x.lo[1] < y.lo[1];
      return x.lo[0] < y.lo[0];
    });
    std::vector<Block> next;
    for (const Merge& m : merges) {
      TreeNode nd;
      nd.index = (int)nodes.size();
      nd.layer = layer;
      nd.axis = axis;
      for (int a = 0; a < 3; ++a) { nd.lo[a] = m.lo[a]; nd.hi[a] = m.hi[a]; }
      const Block& L = blocks[m.left];
      const Block& R = blocks[m.right];
      nd.child_kind[0] = L.kind;
      nd.child[0] = L.id;
      nd.child_kind[1] = R.kind;
      nd.child[1] = R.id;
      nd.sites = L.sites;
      nd.sites.insert(nd.sites.end(), R.sites.begin(), R.sites.end());
      std::sort(nd.sites.begin(), nd.sites.end());
      for (int c = 0; c < 2; ++c)
        if (nd.child_kind[c] == 1) nodes[nd.child[c]].parent = nd.index;
      Block nb;
      nb.kind = 1;
      nb.id = nd.index;
      for (int a = 0; a < 3; ++a) { nb.lo[a] = nd.lo[a]; nb.hi[a] = nd.hi[a]; }
      nb.sites = nd.sites;
      nodes.push_back(nd);
      next.push_back(nb);
    }
    blocks.swap(next);
    ++layer;
    axis = (axis + 1) % 3;
  }
  return nodes;
}

// Node order of one sweep: layers from the bottom (Methods); inside a layer
// a depth-first walk of the tree (first child first), the direction
// alternating between consecutive layers.
std::vector<int> sweep_order(const std::vector<TreeNode>& nodes) {
  const int n = (int)nodes.size();
  std::vector<int> rank(n, 0);
  std::vector<int> stack{n - 1};
  int next = 0;
  while (!stack.empty()) {
    const int i = stack.back();
    stack.pop_back();
    rank[i] = next++;
    for (int c = 1; c >= 0; --c)
      if (nodes[i].child_kind[c] == 1) stack.push_back(nodes[i].child[c]);
  }
  int top = 0;
  for (const TreeNode& t : nodes) top = std::max(top, t.layer);
  std::vector<int> order;
  for (int layer = 0; layer <= top; ++layer) {
    std::vector<int> row;
    for (const TreeNode& t : nodes)
      if (t.layer == layer) row.push_back(t.index);
    std::sort(row.begin(), row.end(), [&](int a, int b) { return rank[a] < rank[b]; });
    if (layer % 2 == 1) std::reverse(row.begin(), row.end());
    order.insert(order.end(), row.begin(), row.end());
  }
  return order;
}

// ---------------------------------------------------------------- sectors
Sectors physical_sectors(int parity) {
  Sectors s;
  if (parity == 1) { s.q = {0, 1}; s.dim = {141, 126}; }
  else { s.q = {-1, 0}; s.dim = {126, 141}; }
  return s;
}

namespace {

// Minimal unsigned big integer (base 2^32) for the exact sector rule.
struct Big {
  std::vector<uint32_t> d;   // little endian, no leading zeros
  Big() {}
  explicit Big(uint64_t v) { while (v) { d.push_back((uint32_t)v); v >>= 32; } }
  bool zero() const { return d.empty(); }
  void trim() { while (!d.empty() && d.back() == 0) d.pop_back(); }
};

Big add(const Big& a, const Big& b) {
  Big r;
  r.d.resize(std::max(a.d.size(), b.d.size()) + 1, 0);
  uint64_t carry = 0;
  for (size_t i = 0; i < r.d.size(); ++i) {
    uint64_t s = carry;
    if (i < a.d.size()) s += a.d[i];
    if (i < b.d.size()) s += b.d[i];
    r.d[i] = (uint32_t)s;
    carry = s >> 32;
  }
  r.trim();
  return r;
}

Big mul(const Big& a, const Big& b) {
  if (a.zero() || b.zero()) return Big();
  std::vector<uint64_t> acc(a.d.size() + b.d.size() + 1, 0);
  Big r;
  r.d.assign(a.d.size() + b.d.size() + 1, 0);
  for (size_t i = 0; i < a.d.size(); ++i) {
    uint64_t carry = 0;
    for (size_t j = 0; j < b.d.size(); ++j) {
      uint64_t cur = (uint64_t)a.d[i] * b.d[j] + r.d[i + j] + carry;
      r.d[i + j] = (uint32_t)cur;
      carry = cur >> 32;
    }
    size_t k = i + b.d.size();
    while (carry) {
      uint64_t cur = (uint64_t)r.d[k] + carry;
      r.d[k] = (uint32_t)cur;
      carry = cur >> 32;
      ++k;
    }
  }
  r.trim();
  return r;
}

int cmp(const Big& a, const Big& b) {
  if (a.d.size() != b.d.size()) return a.d.size() < b.d.size() ? -1 : 1;
  for (size_t i = a.d.size(); i-- > 0;)
    if (a.d[i] != b.d[i]) return a.d[i] < b.d[i] ? -1 : 1;
  return 0;
}

using Dist = std::map<int, Big>;

Dist convolve(const Dist& a, const Dist& b) {
  Dist out;
  for (auto& x : a)
    for (auto& y : b) {
      Big p = mul(x.second, y.second);
      auto it = out.find(x.first + y.first);
      if (it == out.end()) out[x.first + y.first] = p;
      else it->second = add(it->second, p);
    }
  return out;
}

// D(q) for a region with ne even and no odd sites (counts depend only on these).
const Dist& region_counts(int ne, int no) {
  static std::map<std::pair<int, int>, Dist> cache;
  auto key = std::make_pair(ne, no);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  Dist d;
  if (ne == 0 && no == 0) {
    d[0] = Big(1);
  } else if (ne > 0) {
    Dist even;
    even[0] = Big(141);
    even[1] = Big(126);
    d = convolve(region_counts(ne - 1, no), even);
  } else {
    Dist odd;
    odd[-1] = Big(126);
    odd[0] = Big(141);
    d = convolve(region_counts(ne, no - 1), odd);
  }
  return cache[key] = d;
}

Big small(uint64_t v) { return Big(v); }

}  // namespace

bool sector_table(const Params& p, int chi, const std::vector<TreeNode>& nodes, std::vector<Sectors>* bonds,
                  std::string* err) {
  Lattice lat{p.Lx, p.Ly, p.Lz};
  const int N = lat.n_sites();
  int ne_all = 0, no_all = 0;
  for (int s = 0; s < N; ++s) (lat.parity(s) == 1 ? ne_all : no_all)++;
  bonds->assign(nodes.size(), Sectors());
  for (const TreeNode& nd : nodes) {
    std::map<int, int64_t> legs[2];
    for (int c = 0; c < 2; ++c) {
      Sectors s = nd.child_kind[c] == 0 ? physical_sectors(lat.parity(nd.child[c])) : (*bonds)[nd.child[c]];
      for (size_t i = 0; i < s.q.size(); ++i) legs[c][s.q[i]] = s.dim[i];
    }
    std::map<int, int64_t> rows;
    for (auto& a : legs[0])
      for (auto& b : legs[1]) rows[a.first + b.first] += a.second * b.second;
    Sectors out;
    if (nd.parent < 0) {
      if (rows[p.Q] > 0) { out.q = {p.Q}; out.dim = {1}; }
      (*bonds)[nd.index] = out;
      continue;
    }
    int ne = 0, no = 0;
    for (int s : nd.sites) (lat.parity(s) == 1 ? ne : no)++;
    const Dist& dS = region_counts(ne, no);
    const Dist& dC = region_counts(ne_all - ne, no_all - no);
    std::vector<int> qs;
    std::vector<Big> w;
    std::vector<int64_t> cap;
    const Big big_int64(uint64_t(1) << 62);
    for (auto& x : dS) {
      auto itc = dC.find(p.Q - x.first);
      if (itc == dC.end()) continue;
      Big wq = mul(x.second, itc->second);
      int64_t r = rows.count(x.first) ? rows[x.first] : 0;
      // cap = min(D_comp(Q - q), rows_q)
      int64_t c = r;
      if (cmp(itc->second, Big((uint64_t)r)) < 0) {
        c = 0;
        for (size_t i = itc->second.d.size(); i-- > 0;) c = (c << 32) | itc->second.d[i];
      }
      if (wq.zero() || c <= 0) continue;
      qs.push_back(x.first);
      w.push_back(wq);
      cap.push_back(c);
    }
    if (qs.empty()) {
      *err = "empty bond above node " + std::to_string(nd.index);
      return false;
    }
    int64_t capsum = 0;
    for (int64_t c : cap) capsum += c;
    const int64_t chip = std::min<int64_t>(chi, capsum);
    Big W;
    for (const Big& x : w) W = add(W, x);
    const size_t K = qs.size();
    std::vector<Big> num(K);   // chi' * w_q
    std::vector<int64_t> alloc(K, 0);
    for (size_t i = 0; i < K; ++i) {
      num[i] = mul(small((uint64_t)chip), w[i]);
      // floor(num / W): largest f in [0, chi'] with f * W <= num
      int64_t lo = 0, hi = chip;
      while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2;
        if (cmp(mul(small((uint64_t)mid), W), num[i]) <= 0) lo = mid;
        else hi = mid - 1;
      }
      alloc[i] = std::min(lo, cap[i]);
    }
    int64_t missing = chip;
    for (int64_t a : alloc) missing -= a;
    const int n = (int)nd.sites.size();
    while (missing > 0) {
      int best = -1;
      for (size_t i = 0; i < K; ++i) {
        if (alloc[i] >= cap[i]) continue;
        if (best < 0) { best = (int)i; continue; }
        // remainder_i > remainder_best  <=>  num_i + a_best W > num_best + a_i W
        Big lhs = add(num[i], mul(small((uint64_t)alloc[best]), W));
        Big rhs = add(num[best], mul(small((uint64_t)alloc[i]), W));
        int c = cmp(lhs, rhs);
        if (c > 0) { best = (int)i; continue; }
        if (c < 0) continue;
        int64_t di = std::llabs((int64_t)qs[i] * N - (int64_t)p.Q * n);
        int64_t db = std::llabs((int64_t)qs[best] * N - (int64_t)p.Q * n);
        if (di < db || (di == db && qs[i] < qs[best])) best = (int)i;
      }
      if (best < 0) break;
      alloc[best] += 1;
      --missing;
    }
    for (size_t i = 0; i < K; ++i)
      if (alloc[i] > 0) { out.q.push_back(qs[i]); out.dim.push_back((int)alloc[i]); }
    (*bonds)[nd.index] = out;
  }
  // The root's parent leg has dimension one: its child bonds pair up as
  // (q, Q - q); keep the common part of both.
  const TreeNode& root = nodes.back();
  if (root.child_kind[0] == 1 && root.child_kind[1] == 1) {
    Sectors L = (*bonds)[root.child[0]], R = (*bonds)[root.child[1]];
    Sectors nl, nr;
    for (size_t i = 0; i < L.q.size(); ++i) {
      int j = R.find(p.Q - L.q[i]);
      int d = j < 0 ? 0 : std::min(L.dim[i], R.dim[j]);
      if (d > 0) { nl.q.push_back(L.q[i]); nl.dim.push_back(d); }
    }
    for (size_t i = 0; i < R.q.size(); ++i) {
      int j = L.find(p.Q - R.q[i]);
      int d = j < 0 ? 0 : std::min(R.dim[i], L.dim[j]);
      if (d > 0) { nr.q.push_back(R.q[i]); nr.dim.push_back(d); }
    }
    (*bonds)[root.child[0]] = nl;
    (*bonds)[root.child[1]] = nr;
  }
  for (size_t i = 0; i < bonds->size(); ++i)
    if ((*bonds)[i].q.empty()) {
      *err = "empty bond above node " + std::to_string(i);
      return false;
    }
  return true;
}

uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + i * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double splitmix64_uniform(uint64_t raw) {
  return 2.0 * (double)(raw >> 11) * 0x1.0p-53 - 1.0;
}

}  // namespace qed
