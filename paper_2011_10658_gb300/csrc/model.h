// Host-side model of the lattice QED TTN problem: dressed-site basis,
// monomial site operators, lattice geometry, product-term list, binary
// tree and U(1) sector table.  Integer-exact; no GPU code here.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace qed {

constexpr int kLocalDim = 267;   // dressed-site dimension (Methods, after Eq. (14))
constexpr int kHalfLinks = 6;    // -x, -y, -z, +x, +y, +z

// Site-operator kinds.  Half-link indices j, i are 0-based (0..5).
enum OpKind : int {
  OP_IDENTITY = 0,
  OP_M = 1,      // psi^dag eta_j              (Eq. (15), charge +1)
  OP_MD = 2,     // eta_j^dag psi              (Eq. (15), charge -1)
  OP_C = 3,      // eta_i^dag eta_j            (plaquette factor)
  OP_P = 4,      // projector on k_j = k       (Eq. (16))
  OP_N = 5,      // psi^dag psi                (mass term)
  OP_E2 = 6,     // sum over a half-link mask of (1 - k_j)^2 (Eq. (10) squared)
  OP_DIAG = 7,   // arbitrary diagonal (site Hamiltonian)
  OP_PC = 8,     // 1 - projector on k_j = k  (penalty complement)
};

struct OpKey {
  int kind = OP_IDENTITY;
  int a = 0;     // j for M/MD/P, i for C, bit mask for E2
  int b = 0;     // j for C, k for P
  bool operator==(const OpKey& o) const { return kind == o.kind && a == o.a && b == o.b; }
};

// Monomial site operator: (O v)[i] = val[i] * v[src[i]], src = -1 for a zero row.
struct SiteOp {
  int16_t src[kLocalDim];
  double val[kLocalDim];
  int dq = 0;    // charge shift: q(out) - q(in)
};

struct Params {
  int32_t Lx = 2, Ly = 2, Lz = 2;
  int32_t boundary = 0;          // 0 = open with dangling half-links, 1 = periodic
  // local chemical potentials mu_x (one per site, empty = none): terms
  // mu_x psi^dag_x psi_x of their own class (Methods: the diagonal local
  // terms used to pin charges)
  std::vector<double> mu;
  double t = 1.0, m = 1.0, ge2 = 1.0, cB = 0.5, nu = 10.0;
  int32_t Q = 0;
};

// Coupling classes, in the order t, m, ge2, cB, nu.
// N_COUPLINGS scalar couplings; the chemical potentials form one more class.
enum CouplingClass : int { CLS_T = 0, CLS_M = 1, CLS_GE2 = 2, CLS_CB = 3, CLS_NU = 4, CLS_MU = 5, N_CLASSES = 6 };
constexpr int N_COUPLINGS = 5;

struct Term {
  double coef = 0.0;
  int cls = 0;
  std::vector<std::pair<int, OpKey>> ops;  // (site, op) sorted by site
};

// Basis row: phi, k1..k6, sign, q (int8 each); 267 rows per parity.
void enumerate_basis(int parity, int8_t* table /* [267][9] */);
int site_charge(int parity, int row);
void build_site_op(int parity, const OpKey& key, SiteOp* out);

struct Lattice {
  int Lx, Ly, Lz;
  // 1: periodic in every direction with more than one site (a direction of
  // extent 1 has no links and keeps its dangling half-links)
  int periodic = 0;
  int n_sites() const { return Lx * Ly * Lz; }
  int index(int i, int j, int k) const { return i + Lx * (j + Ly * k); }
  void coords(int s, int c[3]) const;
  int parity(int s) const;
  int neighbour(int s, int mu, int step) const;   // -1 if outside
  std::vector<int> dangling(int s) const;
  int electric_mask(int s) const;                 // bit mask over half-links
  int n_links() const;
};

void build_terms(const Params& p, std::vector<Term>* terms, double* constant);

struct TreeNode {
  int index = 0, layer = 0, axis = 0;
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  int child_kind[2] = {0, 0};   // 0 = site, 1 = node
  int child[2] = {0, 0};
  int parent = -1;
  std::vector<int> sites;       // sorted
};

std::vector<TreeNode> build_tree(int Lx, int Ly, int Lz);
// Order of the node updates in one sweep (layers bottom-up, depth-first
// inside a layer, direction alternating per layer).
std::vector<int> sweep_order(const std::vector<TreeNode>& nodes);

// Sector list of a bond: ascending charges with dimensions.
struct Sectors {
  std::vector<int> q;
  std::vector<int> dim;
  int total() const { int s = 0; for (int d : dim) s += d; return s; }
  int find(int charge) const { for (size_t i = 0; i < q.size(); ++i) if (q[i] == charge) return (int)i; return -1; }
  int offset(int idx) const { int s = 0; for (int i = 0; i < idx; ++i) s += dim[i]; return s; }
};

Sectors physical_sectors(int parity);
// Bond sectors above every node (root: {Q: 1}).  Returns false with a
// message if some bond comes out empty.
bool sector_table(const Params& p, int chi, const std::vector<TreeNode>& nodes,
                  std::vector<Sectors>* bonds, std::string* err);

// SplitMix64 (Steele, Lea & Flood 2014): output number i (1-based) of the
// stream seeded with seed.
uint64_t splitmix64_at(uint64_t seed, uint64_t i);
double splitmix64_uniform(uint64_t raw);   // 2 * (x >> 11) * 2^-53 - 1

}  // namespace qed
