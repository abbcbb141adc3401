// Symmetry labels, the Fermi-Hubbard MPO and FP64 recoupling coefficients.
//
// Sec. S2.1 (Eq. symdecomp): every bond space is a direct sum of multiplets
// labelled by a U(1) charge and an SU(2) spin, with a degeneracy d per label;
// tensors are stored as one reduced block per allowed label combination.  The
// engine works in the particle-hole (Shiba) frame c_{i dn} -> (-1)^i c^dag_{i dn},
// where the charge SU(2) of the paper becomes the ordinary spin SU(2) and the
// Neel state becomes the spin-singlet product |2,0,2,0,...>.  Two symmetry modes
// share every code path:
//   U1U1 : labels (n, 2 S^z), every multiplet one-dimensional;
//   U1SU2: labels (n, 2 S),   multiplets of dimension 2S+1 (reduced tensors).
// Recoupling coefficients are computed numerically in FP64 by contracting the
// Clebsch-Gordan structure tensors of the inputs with the m-resolved MPO and
// projecting onto the output's fusion-tree basis; U1U1 is the special case in
// which every structure tensor is the scalar 1.
#pragma once
#include <array>
#include <cstdint>
#include <map>
#include <mutex>
#include <unordered_map>
#include <vector>

namespace tdvp {

struct Mult {
  int n, t;                // U(1) charge and t = 2S (SU(2)) or 2S^z (U1U1)
  int tj;                  // 2j used for Clebsch-Gordan coefficients (0 in U1U1)
  std::vector<int> comps;  // components in the m-resolved basis, m = +j first
};

struct Sector {
  int n, t, d;
};

struct BondSpace {
  std::vector<Sector> s;
  std::unordered_map<uint64_t, int> idx;  // (n, t) packed as key(n, t) -> sector index
  static uint64_t key(int n, int t) { return ((uint64_t)(uint32_t)n << 32) | (uint32_t)t; }
  void build_index();
  int find(int n, int t) const;
  long long chi_red() const;   // sum d
  int dmax() const;
};

struct Model {
  bool su2 = false;
  double J = 1.0, U = 0.0;
  std::vector<Mult> site;  // local multiplets (3 in SU(2), 4 in U1U1)
  std::vector<Mult> chan;  // MPO channel multiplets (4 in SU(2), 6 in U1U1)
  int chB = 0, chE = 0;    // channel multiplet indices of the B ("nothing yet") and E ("done") rows
  double W[6][6][4][4];    // m-resolved bulk MPO W[w][w'][s'][s] = <s'| W_{w w'} |s>
  double occ_n[4], occ_up[4], occ_dn[4], occ_d[4];  // per site multiplet, in the engine frame

  void init(bool su2, double J, double U);
  // labels of q1 x q2
  void fuse(int n1, int t1, int n2, int t2, std::vector<std::pair<int, int>>& out) const;
  int mult_dim(int t) const { return su2 ? t + 1 : 1; }
  int tj_of(int t) const { return su2 ? t : 0; }
};

// Exact-as-possible Clebsch-Gordan <j1 m1; j2 m2 | J M> (all doubled), Racah formula.
double clebsch(int tj1, int tm1, int tj2, int tm2, int tJ, int tM);
// Cached array C[m1][m2][M] (m index 0 = +j), row-major (tj1+1)(tj2+1)(tJ+1).
const std::vector<double>& cg_array(int tj1, int tj2, int tJ);

// Output entry of a recoupling: which output tree and the FP64 coefficient.
struct Recouple2 {  // two-site H_eff step 2: T1(a',w,a,s1,c,s2,b) -> T2(a',s1',c',s2',b',w2,b)
  int s1p, tcp, s2p, tbp, w2;
  double f;
};
struct Recouple1 {  // one-site H_eff / left-env step 2: T1(a',w,a,s,b) -> T2(a',s',b'',w',b)
  int sp, tbpp, wp;
  double f;
};
struct RecoupleR {  // right-env step 2: F1(a,s,b,w',b') -> F2(a,w,a'',s',b')
  int w, tapp, sp;
  double f;
};

class Recoupler {
 public:
  explicit Recoupler(const Model* m) : m_(m) {}
  const std::vector<Recouple2>& two_site(int tap, int w, int ta, int s1, int tc, int s2, int tb);
  const std::vector<Recouple1>& one_site(int tap, int w, int ta, int s, int tb);
  const std::vector<RecoupleR>& right_env(int ta, int s, int tb, int wp, int tbp);

 private:
  const Model* m_;
  std::mutex mu_;
  std::unordered_map<uint64_t, std::vector<Recouple2>> c2_;
  std::unordered_map<uint64_t, std::vector<Recouple1>> c1_;
  std::unordered_map<uint64_t, std::vector<RecoupleR>> cr_;
};

}  // namespace tdvp
