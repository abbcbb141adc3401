// Symmetry labels, the Fermi-Hubbard MPO in the particle-hole frame, and FP64
// recoupling coefficients (see sym.hpp).
#include "sym.hpp"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace tdvp {

// ---------------------------------------------------------------------------
// bond spaces
// ---------------------------------------------------------------------------

void BondSpace::build_index() {
  idx.clear();
  idx.reserve(2 * s.size() + 1);
  for (int k = 0; k < (int)s.size(); ++k) idx[key(s[k].n, s[k].t)] = k;
}

int BondSpace::find(int n, int t) const {
  auto it = idx.find(key(n, t));
  return it == idx.end() ? -1 : it->second;
}

long long BondSpace::chi_red() const {
  long long c = 0;
  for (auto& x : s) c += x.d;
  return c;
}

int BondSpace::dmax() const {
  int m = 0;
  for (auto& x : s) m = std::max(m, x.d);
  return m;
}

// ---------------------------------------------------------------------------
// Clebsch-Gordan coefficients: Racah's closed form in long double
// ---------------------------------------------------------------------------

static long double fact_h(int n2) {  // (n2/2)!
  long double r = 1;
  for (int k = 2; k <= n2 / 2; ++k) r *= k;
  return r;
}

double clebsch(int tj1, int tm1, int tj2, int tm2, int tJ, int tM) {
  if (tm1 + tm2 != tM) return 0.0;
  if (tJ < std::abs(tj1 - tj2) || tJ > tj1 + tj2 || ((tj1 + tj2 + tJ) & 1)) return 0.0;
  if (std::abs(tm1) > tj1 || std::abs(tm2) > tj2 || std::abs(tM) > tJ) return 0.0;
  if (((tj1 + tm1) & 1) || ((tj2 + tm2) & 1) || ((tJ + tM) & 1)) return 0.0;
  long double pref = (tJ + 1) * fact_h(tJ + tj1 - tj2) * fact_h(tJ - tj1 + tj2) * fact_h(tj1 + tj2 - tJ) /
                     fact_h(tj1 + tj2 + tJ + 2);
  pref *= fact_h(tJ + tM) * fact_h(tJ - tM) * fact_h(tj1 - tm1) * fact_h(tj1 + tm1) * fact_h(tj2 - tm2) *
          fact_h(tj2 + tm2);
  long double sum = 0;
  for (int k = 0;; ++k) {
    int a0 = tj1 + tj2 - tJ - 2 * k, a1 = tj1 - tm1 - 2 * k, a2 = tj2 + tm2 - 2 * k;
    int a3 = tJ - tj2 + tm1 + 2 * k, a4 = tJ - tj1 - tm2 + 2 * k;
    if (a0 < 0 || a1 < 0 || a2 < 0) break;
    if (a3 < 0 || a4 < 0) continue;
    long double den = fact_h(2 * k) * fact_h(a0) * fact_h(a1) * fact_h(a2) * fact_h(a3) * fact_h(a4);
    sum += ((k & 1) ? -1.0L : 1.0L) / den;
  }
  return (double)(std::sqrt(pref) * sum);
}

const std::vector<double>& cg_array(int tj1, int tj2, int tJ) {
  static std::mutex mu;
  static std::map<std::array<int, 3>, std::vector<double>> cache;
  std::lock_guard<std::mutex> g(mu);
  auto key = std::array<int, 3>{tj1, tj2, tJ};
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  std::vector<double> C((tj1 + 1) * (tj2 + 1) * (tJ + 1));
  for (int a = 0; a <= tj1; ++a)
    for (int b = 0; b <= tj2; ++b)
      for (int c = 0; c <= tJ; ++c)
        C[(a * (tj2 + 1) + b) * (tJ + 1) + c] = clebsch(tj1, tj1 - 2 * a, tj2, tj2 - 2 * b, tJ, tJ - 2 * c);
  return cache.emplace(key, std::move(C)).first->second;
}

// ---------------------------------------------------------------------------
// model: local operators and the particle-hole-frame MPO
// ---------------------------------------------------------------------------

namespace {
using M4 = std::array<std::array<double, 4>, 4>;
M4 zero4() {
  M4 m{};
  return m;
}
M4 mul(const M4& a, const M4& b) {
  M4 r = zero4();
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      for (int k = 0; k < 4; ++k) r[i][j] += a[i][k] * b[k][j];
  return r;
}
M4 tr(const M4& a) {
  M4 r = zero4();
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) r[i][j] = a[j][i];
  return r;
}
}  // namespace

void Model::init(bool su2_, double J_, double U_) {
  su2 = su2_;
  J = J_;
  U = U_;
  // site basis index s = n_up + 2 n_dn; up is the lower fermion mode inside a site
  M4 a_up = zero4(), a_dn = zero4(), F = zero4(), I = zero4();
  for (int s = 0; s < 4; ++s) {
    int nu = s & 1, nd = (s >> 1) & 1;
    F[s][s] = ((nu + nd) & 1) ? -1.0 : 1.0;
    I[s][s] = 1.0;
    if (nu) a_up[s - 1][s] = 1.0;
    if (nd) a_dn[s - 2][s] = nu ? -1.0 : 1.0;
  }
  M4 n_up = mul(tr(a_up), a_up), n_dn = mul(tr(a_dn), a_dn);
  for (int w = 0; w < 6; ++w)
    for (int v = 0; v < 6; ++v)
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) W[w][v][a][b] = 0.0;
  auto set = [&](int w, int v, const M4& m, double f) {
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) W[w][v][a][b] = f * m[a][b];
  };
  // channels: 0 B, 1 cd(+1/2), 2 cd(-1/2), 3 c(+1/2), 4 c(-1/2), 5 E
  set(0, 0, I, 1.0);
  set(5, 5, I, 1.0);
  M4 onsite = zero4();
  M4 nn = mul(n_up, n_dn);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) onsite[a][b] = -U * nn[a][b] + 0.5 * U * (n_up[a][b] + n_dn[a][b]);
  set(0, 5, onsite, 1.0);
  set(0, 1, mul(tr(a_up), F), -J);
  set(1, 5, a_up, 1.0);
  set(0, 2, mul(tr(a_dn), F), -J);
  set(2, 5, a_dn, 1.0);
  set(0, 3, mul(F, a_dn), -J);
  set(3, 5, tr(a_dn), 1.0);
  set(0, 4, mul(F, a_up), J);
  set(4, 5, tr(a_up), -1.0);

  site.clear();
  chan.clear();
  if (su2) {
    site = {{0, 0, 0, {0}}, {1, 1, 1, {1, 2}}, {2, 0, 0, {3}}};
    chan = {{0, 0, 0, {0}}, {1, 1, 1, {1, 2}}, {-1, 1, 1, {3, 4}}, {0, 0, 0, {5}}};
    chB = 0;
    chE = 3;
    double n[3] = {0, 1, 2}, d[3] = {0, 0, 1};
    for (int k = 0; k < 3; ++k) {
      occ_n[k] = n[k];
      occ_up[k] = 0.5 * n[k];
      occ_dn[k] = 0.5 * n[k];
      occ_d[k] = d[k];
    }
  } else {
    site = {{0, 0, 0, {0}}, {1, 1, 0, {1}}, {1, -1, 0, {2}}, {2, 0, 0, {3}}};
    chan = {{0, 0, 0, {0}}, {1, 1, 0, {1}}, {1, -1, 0, {2}}, {-1, 1, 0, {3}}, {-1, -1, 0, {4}}, {0, 0, 0, {5}}};
    chB = 0;
    chE = 5;
    double up[4] = {0, 1, 0, 1}, dn[4] = {0, 0, 1, 1};
    for (int k = 0; k < 4; ++k) {
      occ_up[k] = up[k];
      occ_dn[k] = dn[k];
      occ_n[k] = up[k] + dn[k];
      occ_d[k] = up[k] * dn[k];
    }
  }
}

void Model::fuse(int n1, int t1, int n2, int t2, std::vector<std::pair<int, int>>& out) const {
  out.clear();
  if (su2) {
    for (int t = std::abs(t1 - t2); t <= t1 + t2; t += 2) out.push_back({n1 + n2, t});
  } else {
    out.push_back({n1 + n2, t1 + t2});
  }
}

// ---------------------------------------------------------------------------
// recoupling coefficients
// ---------------------------------------------------------------------------

namespace {

inline uint64_t pack(std::initializer_list<int> v) {
  uint64_t k = 0;
  for (int x : v) k = (k << 8) | (uint64_t)((x + 128) & 0xff);
  return k;
}

// small dense tensor with row-major strides
struct T5 {
  int d[5];
  std::vector<double> v;
  T5(int a, int b, int c, int e, int f) : d{a, b, c, e, f}, v((size_t)a * b * c * e * f, 0.0) {}
  double& operator()(int i, int j, int k, int l, int m) {
    return v[((((size_t)i * d[1] + j) * d[2] + k) * d[3] + l) * d[4] + m];
  }
};

inline double C3(const std::vector<double>& c, int tj2, int tJ, int a, int b, int m) {
  return c[((size_t)a * (tj2 + 1) + b) * (tJ + 1) + m];
}

bool contains(const std::vector<std::pair<int, int>>& v, int t) {
  for (auto& p : v)
    if (p.second == t) return true;
  return false;
}

}  // namespace

const std::vector<Recouple2>& Recoupler::two_site(int tap, int w, int ta, int s1, int tc, int s2, int tb) {
  uint64_t key = pack({tap, w, ta, s1, tc, s2, tb});
  {
    std::lock_guard<std::mutex> g(mu_);
    auto it = c2_.find(key);
    if (it != c2_.end()) return it->second;
  }
  const Model& M = *m_;
  const Mult &mw = M.chan[w], &m1 = M.site[s1], &m2 = M.site[s2];
  int jap = M.tj_of(tap), ja = M.tj_of(ta), jc = M.tj_of(tc), jb = M.tj_of(tb);
  int jw = mw.tj, j1 = m1.tj, j2 = m2.tj;
  const auto& cL = cg_array(ja, jw, jap);
  const auto& cA = cg_array(ja, j1, jc);
  const auto& cB = cg_array(jc, j2, jb);
  // X_T1[a', mu, s1, s2, b] = sum_alpha C(a w|a') sum_gamma C(a s1|c) C(c s2|b)
  T5 X(jap + 1, jw + 1, j1 + 1, j2 + 1, jb + 1);
  for (int al = 0; al <= ja; ++al)
    for (int mu = 0; mu <= jw; ++mu)
      for (int alp = 0; alp <= jap; ++alp) {
        double l = C3(cL, jw, jap, al, mu, alp);
        if (l == 0.0) continue;
        for (int x1 = 0; x1 <= j1; ++x1)
          for (int g = 0; g <= jc; ++g) {
            double a = C3(cA, j1, jc, al, x1, g);
            if (a == 0.0) continue;
            for (int x2 = 0; x2 <= j2; ++x2)
              for (int be = 0; be <= jb; ++be) X(alp, mu, x1, x2, be) += l * a * C3(cB, j2, jb, g, x2, be);
          }
      }
  std::vector<Recouple2> out;
  std::vector<std::pair<int, int>> fc, fb, fw;
  for (int w2 = 0; w2 < (int)M.chan.size(); ++w2) {
    const Mult& mw2 = M.chan[w2];
    int jw2 = mw2.tj;
    for (int s1p = 0; s1p < (int)M.site.size(); ++s1p)
      for (int s2p = 0; s2p < (int)M.site.size(); ++s2p) {
        const Mult &m1p = M.site[s1p], &m2p = M.site[s2p];
        int j1p = m1p.tj, j2p = m2p.tj;
        // Wpair[mu][x1'][x1][x2'][x2][mu2]
        bool any = false;
        std::vector<double> Wp((size_t)(jw + 1) * (j1p + 1) * (j1 + 1) * (j2p + 1) * (j2 + 1) * (jw2 + 1), 0.0);
        auto wi = [&](int mu, int y1, int x1, int y2, int x2, int mu2) {
          return ((((((size_t)mu * (j1p + 1) + y1) * (j1 + 1) + x1) * (j2p + 1) + y2) * (j2 + 1) + x2) * (jw2 + 1) +
                  mu2);
        };
        for (int mu = 0; mu <= jw; ++mu)
          for (int y1 = 0; y1 <= j1p; ++y1)
            for (int x1 = 0; x1 <= j1; ++x1)
              for (int y2 = 0; y2 <= j2p; ++y2)
                for (int x2 = 0; x2 <= j2; ++x2)
                  for (int mu2 = 0; mu2 <= jw2; ++mu2) {
                    double s = 0.0;
                    for (int xx = 0; xx < 6; ++xx)
                      s += M.W[mw.comps[mu]][xx][m1p.comps[y1]][m1.comps[x1]] *
                           M.W[xx][mw2.comps[mu2]][m2p.comps[y2]][m2.comps[x2]];
                    if (s != 0.0) any = true;
                    Wp[wi(mu, y1, x1, y2, x2, mu2)] = s;
                  }
        if (!any) continue;
        // Y[a', y1, y2, mu2, b]
        T5 Y(jap + 1, j1p + 1, j2p + 1, jw2 + 1, jb + 1);
        for (int alp = 0; alp <= jap; ++alp)
          for (int mu = 0; mu <= jw; ++mu)
            for (int x1 = 0; x1 <= j1; ++x1)
              for (int x2 = 0; x2 <= j2; ++x2)
                for (int be = 0; be <= jb; ++be) {
                  double xv = X(alp, mu, x1, x2, be);
                  if (xv == 0.0) continue;
                  for (int y1 = 0; y1 <= j1p; ++y1)
                    for (int y2 = 0; y2 <= j2p; ++y2)
                      for (int mu2 = 0; mu2 <= jw2; ++mu2) {
                        double wv = Wp[wi(mu, y1, x1, y2, x2, mu2)];
                        if (wv != 0.0) Y(alp, y1, y2, mu2, be) += xv * wv;
                      }
                }
        // project on every output tree (c', b') with b' in b x w2
        M.fuse(0, tap, 0, m1p.t, fc);
        M.fuse(0, tb, 0, mw2.t, fw);
        for (auto& pc : fc) {
          int tcp = pc.second, jcp = M.tj_of(tcp);
          M.fuse(0, tcp, 0, m2p.t, fb);
          for (auto& pb : fb) {
            int tbp = pb.second;
            if (!contains(fw, tbp)) continue;
            int jbp = M.tj_of(tbp);
            const auto& d1 = cg_array(jap, j1p, jcp);
            const auto& d2 = cg_array(jcp, j2p, jbp);
            const auto& d3 = cg_array(jb, jw2, jbp);
            double num = 0.0, den = 0.0;
            for (int alp = 0; alp <= jap; ++alp)
              for (int y1 = 0; y1 <= j1p; ++y1)
                for (int y2 = 0; y2 <= j2p; ++y2)
                  for (int mu2 = 0; mu2 <= jw2; ++mu2)
                    for (int be = 0; be <= jb; ++be) {
                      double xt = 0.0;
                      for (int gp = 0; gp <= jcp; ++gp) {
                        double a = C3(d1, j1p, jcp, alp, y1, gp);
                        if (a == 0.0) continue;
                        for (int bp = 0; bp <= jbp; ++bp)
                          xt += a * C3(d2, j2p, jbp, gp, y2, bp) * C3(d3, jw2, jbp, be, mu2, bp);
                      }
                      num += xt * Y(alp, y1, y2, mu2, be);
                      den += xt * xt;
                    }
            if (den == 0.0) continue;
            double f = num / den;
            if (std::fabs(f) > 1e-13) out.push_back({s1p, tcp, s2p, tbp, w2, f});
          }
        }
      }
  }
  std::lock_guard<std::mutex> g(mu_);
  return c2_.emplace(key, std::move(out)).first->second;
}

const std::vector<Recouple1>& Recoupler::one_site(int tap, int w, int ta, int s, int tb) {
  uint64_t key = pack({tap, w, ta, s, tb});
  {
    std::lock_guard<std::mutex> g(mu_);
    auto it = c1_.find(key);
    if (it != c1_.end()) return it->second;
  }
  const Model& M = *m_;
  const Mult &mw = M.chan[w], &ms = M.site[s];
  int jap = M.tj_of(tap), ja = M.tj_of(ta), jb = M.tj_of(tb), jw = mw.tj, js = ms.tj;
  const auto& cL = cg_array(ja, jw, jap);
  const auto& cA = cg_array(ja, js, jb);
  // X[a', mu, s, b, 1]
  T5 X(jap + 1, jw + 1, js + 1, jb + 1, 1);
  for (int al = 0; al <= ja; ++al)
    for (int mu = 0; mu <= jw; ++mu)
      for (int alp = 0; alp <= jap; ++alp) {
        double l = C3(cL, jw, jap, al, mu, alp);
        if (l == 0.0) continue;
        for (int x = 0; x <= js; ++x)
          for (int be = 0; be <= jb; ++be) X(alp, mu, x, be, 0) += l * C3(cA, js, jb, al, x, be);
      }
  std::vector<Recouple1> out;
  std::vector<std::pair<int, int>> f1, f2;
  for (int wp = 0; wp < (int)M.chan.size(); ++wp) {
    const Mult& mwp = M.chan[wp];
    int jwp = mwp.tj;
    for (int sp = 0; sp < (int)M.site.size(); ++sp) {
      const Mult& msp = M.site[sp];
      int jsp = msp.tj;
      T5 Y(jap + 1, jsp + 1, jwp + 1, jb + 1, 1);
      bool any = false;
      for (int alp = 0; alp <= jap; ++alp)
        for (int mu = 0; mu <= jw; ++mu)
          for (int x = 0; x <= js; ++x)
            for (int be = 0; be <= jb; ++be) {
              double xv = X(alp, mu, x, be, 0);
              if (xv == 0.0) continue;
              for (int y = 0; y <= jsp; ++y)
                for (int mp = 0; mp <= jwp; ++mp) {
                  double wv = M.W[mw.comps[mu]][mwp.comps[mp]][msp.comps[y]][ms.comps[x]];
                  if (wv != 0.0) {
                    Y(alp, y, mp, be, 0) += xv * wv;
                    any = true;
                  }
                }
            }
      if (!any) continue;
      M.fuse(0, tap, 0, msp.t, f1);
      M.fuse(0, tb, 0, mwp.t, f2);
      for (auto& p : f1) {
        int tbpp = p.second;
        if (!contains(f2, tbpp)) continue;
        int jbpp = M.tj_of(tbpp);
        const auto& d1 = cg_array(jap, jsp, jbpp);
        const auto& d2 = cg_array(jb, jwp, jbpp);
        double num = 0.0, den = 0.0;
        for (int alp = 0; alp <= jap; ++alp)
          for (int y = 0; y <= jsp; ++y)
            for (int mp = 0; mp <= jwp; ++mp)
              for (int be = 0; be <= jb; ++be) {
                double xt = 0.0;
                for (int bpp = 0; bpp <= jbpp; ++bpp)
                  xt += C3(d1, jsp, jbpp, alp, y, bpp) * C3(d2, jwp, jbpp, be, mp, bpp);
                num += xt * Y(alp, y, mp, be, 0);
                den += xt * xt;
              }
        if (den == 0.0) continue;
        double f = num / den;
        if (std::fabs(f) > 1e-13) out.push_back({sp, tbpp, wp, f});
      }
    }
  }
  std::lock_guard<std::mutex> g(mu_);
  return c1_.emplace(key, std::move(out)).first->second;
}

const std::vector<RecoupleR>& Recoupler::right_env(int ta, int s, int tb, int wp, int tbp) {
  uint64_t key = pack({ta, s, tb, wp, tbp});
  {
    std::lock_guard<std::mutex> g(mu_);
    auto it = cr_.find(key);
    if (it != cr_.end()) return it->second;
  }
  const Model& M = *m_;
  const Mult &ms = M.site[s], &mwp = M.chan[wp];
  int ja = M.tj_of(ta), jb = M.tj_of(tb), jbp = M.tj_of(tbp), js = ms.tj, jwp = mwp.tj;
  const auto& cA = cg_array(ja, js, jb);
  const auto& cR = cg_array(jb, jwp, jbp);
  // X_F1[a, s, mu', b'] = sum_beta C(a s|b) C(b w'|b')
  T5 X(ja + 1, js + 1, jwp + 1, jbp + 1, 1);
  for (int al = 0; al <= ja; ++al)
    for (int x = 0; x <= js; ++x)
      for (int be = 0; be <= jb; ++be) {
        double a = C3(cA, js, jb, al, x, be);
        if (a == 0.0) continue;
        for (int mp = 0; mp <= jwp; ++mp)
          for (int bp = 0; bp <= jbp; ++bp) X(al, x, mp, bp, 0) += a * C3(cR, jwp, jbp, be, mp, bp);
      }
  std::vector<RecoupleR> out;
  std::vector<std::pair<int, int>> f1;
  for (int w = 0; w < (int)M.chan.size(); ++w) {
    const Mult& mw = M.chan[w];
    int jw = mw.tj;
    for (int sp = 0; sp < (int)M.site.size(); ++sp) {
      const Mult& msp = M.site[sp];
      int jsp = msp.tj;
      // Y[a, mu, s', b']
      T5 Y(ja + 1, jw + 1, jsp + 1, jbp + 1, 1);
      bool any = false;
      for (int al = 0; al <= ja; ++al)
        for (int x = 0; x <= js; ++x)
          for (int mp = 0; mp <= jwp; ++mp)
            for (int bp = 0; bp <= jbp; ++bp) {
              double xv = X(al, x, mp, bp, 0);
              if (xv == 0.0) continue;
              for (int mu = 0; mu <= jw; ++mu)
                for (int y = 0; y <= jsp; ++y) {
                  double wv = M.W[mw.comps[mu]][mwp.comps[mp]][msp.comps[y]][ms.comps[x]];
                  if (wv != 0.0) {
                    Y(al, mu, y, bp, 0) += xv * wv;
                    any = true;
                  }
                }
            }
      if (!any) continue;
      M.fuse(0, ta, 0, mw.t, f1);
      for (auto& p : f1) {
        int tapp = p.second;
        std::vector<std::pair<int, int>> f2;
        M.fuse(0, tapp, 0, msp.t, f2);
        if (!contains(f2, tbp)) continue;
        int japp = M.tj_of(tapp);
        const auto& d1 = cg_array(ja, jw, japp);
        const auto& d2 = cg_array(japp, jsp, jbp);
        double num = 0.0, den = 0.0;
        for (int al = 0; al <= ja; ++al)
          for (int mu = 0; mu <= jw; ++mu)
            for (int y = 0; y <= jsp; ++y)
              for (int bp = 0; bp <= jbp; ++bp) {
                double xt = 0.0;
                for (int app = 0; app <= japp; ++app)
                  xt += C3(d1, jw, japp, al, mu, app) * C3(d2, jsp, jbp, app, y, bp);
                num += xt * Y(al, mu, y, bp, 0);
                den += xt * xt;
              }
        if (den == 0.0) continue;
        double f = num / den;
        if (std::fabs(f) > 1e-13) out.push_back({w, tapp, sp, f});
      }
    }
  }
  std::lock_guard<std::mutex> g(mu_);
  return cr_.emplace(key, std::move(out)).first->second;
}

}  // namespace tdvp
