// Plain, slow FP64 CPU oracle of the multilevel octree lattice Boltzmann method
// of Qi, Klimach & Roller, "Implementation of the compact interpolation within
// the octree based Lattice Boltzmann solver Musubi" (arXiv:1601.06984).
//
// TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library against
// an independent statement of the method.  It shares no code, header, table or
// helper with the CUDA path; only tests/, the smoke check and the bench's CPU
// baseline leg load it.  Nothing in the product path may call it.
//
// Every quantity is computed in the most direct way the paper states it: per
// level hash maps keyed by integer coordinates, one element at a time, scalar
// loops over the discrete velocities.  The loops over the elements of a level
// may be spread over OpenMP threads (orc_set_threads); each element's
// arithmetic is the same either way, and the sums over elements (reductions)
// stay sequential, so the results do not depend on the thread count.  The scalar type T is double or a
// forward-mode dual number (value, tangent) so that directional derivatives of
// any output can be taken exactly; that is what the adjoint is checked against.
//
// What follows which passage of the paper:
//   lattice BGK update ............. Sec. 2.1, Eqs. (lbe), (bgk)
//   equilibrium .................... Sec. 2.1, Eq. (feq) with the sign of the
//                                    u.u term taken as minus (the printed plus
//                                    breaks sum_i f^eq_i = rho)
//   moments, viscosity, strain ..... Sec. 2.1, Eq. (nu) and the strain-rate eq.
//   levels, acoustic scaling,
//   relaxation scaling ............. Sec. 2.2, Eq. (fneq_scale)
//   ghost kinds GFC / GFF .......... Sec. 2.2
//   compact quadratic velocity ..... Sec. 2.2, Eqs. (compact_3D_u), (compact_3D_s);
//                                    2D: the same construction on the unit
//                                    square (the paper only cites Geier 2009)
//   interpolation steps 1-5 ........ Sec. 2.2 (enumerated steps); the f^neq
//                                    rescale includes the factor 1/m implied by
//                                    acoustic scaling and the strain-rate eq.
//   GFF before GFC, two ghost layers  Sec. 2.2 (closing paragraphs)
//   diffusive scaling, four layers . Sec. 2.2 (named there only; time-step
//                                    ratio 4, omega equal on all levels and
//                                    the unit conversions are readings)
//   inlet / outlet / wall / force .. Sec. 2.3
//   treeID, z-curve, weights ....... Sec. 3.1, Eq. (weight)
//   initial f^neq .................. Sec. 4.1 (prefactor chosen so that the
//                                    strain-rate eq. returns S exactly)
// Readings where the paper is silent (Guo forcing, post-collision storage,
// linear-in-time ghost refill, outlet index mapping, GFF averaging weights)
// are stated where they are used.

#include <algorithm>
#include <type_traits>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v = 0.0, d = 0.0;
  Dual() = default;
  Dual(double a) : v(a), d(0.0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, Dual b) { return a = a + b; }
inline Dual& operator-=(Dual& a, Dual b) { return a = a - b; }
inline double value_of(double x) { return x; }
inline double value_of(const Dual& x) { return x.v; }
inline double tangent_of(double) { return 0.0; }
inline double tangent_of(const Dual& x) { return x.d; }

// ---------------------------------------------------------------- lattices
// Discrete velocities and weights (Sec. 2.1; the paper names the lattices and
// cites Qian et al. for them).  Direction order, also used by the user-facing
// per-direction arrays:
//   D2Q9 : 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 (+x+y), 6 (-x-y), 7 (+x-y), 8 (-x+y)
//   D3Q19: 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z,
//          7 (+x+y), 8 (-x-y), 9 (+x-y), 10 (-x+y),
//          11 (+x+z), 12 (-x-z), 13 (+x-z), 14 (-x+z),
//          15 (+y+z), 16 (-y-z), 17 (+y-z), 18 (-y+z)
//   D3Q27: the D3Q19 set, then 19 (+x+y+z), 20 (-x-y-z), 21 (+x+y-z),
//          22 (-x-y+z), 23 (+x-y+z), 24 (-x+y-z), 25 (-x+y+z), 26 (+x-y-z)
// Weights by |c|^2 (Sec. 2.1 uses the standard D2Q9 / D3Q19 / D3Q27 sets):
//   D2Q9 4/9, 1/9, 1/36;  D3Q19 1/3, 1/18, 1/36;  D3Q27 8/27, 2/27, 1/54, 1/216.
constexpr int kQmax = 27;
// element loops shorter than this stay on one thread (thread start-up would
// cost more than the loop)
constexpr int64_t kParMin = 4096;
struct Lattice {
  int d = 0, Q = 0;
  int c[kQmax][3] = {};
  double w[kQmax] = {};
  int opp[kQmax] = {};
};

Lattice make_lattice(int q) {
  Lattice lat;
  if (q == 9) {
    lat.d = 2;
    lat.Q = 9;
    const int cc[9][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1},
                          {1, 1}, {-1, -1}, {1, -1}, {-1, 1}};
    for (int i = 0; i < 9; ++i) {
      lat.c[i][0] = cc[i][0];
      lat.c[i][1] = cc[i][1];
      lat.c[i][2] = 0;
      int n2 = cc[i][0] * cc[i][0] + cc[i][1] * cc[i][1];
      lat.w[i] = n2 == 0 ? 4.0 / 9.0 : (n2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
  } else {
    lat.d = 3;
    lat.Q = q;
    const int cc[27][3] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},
                           {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},  {1, 0, 1},
                           {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},  {0, 1, 1},   {0, -1, -1}, {0, 1, -1},
                           {0, -1, 1},  {1, 1, 1},   {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1}, {1, -1, 1},
                           {-1, 1, -1}, {-1, 1, 1},  {1, -1, -1}};
    for (int i = 0; i < q; ++i) {
      int n2 = 0;
      for (int a = 0; a < 3; ++a) {
        lat.c[i][a] = cc[i][a];
        n2 += cc[i][a] * cc[i][a];
      }
      if (q == 19) lat.w[i] = n2 == 0 ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
      else lat.w[i] = n2 == 0 ? 8.0 / 27.0 : (n2 == 1 ? 2.0 / 27.0 : (n2 == 2 ? 1.0 / 54.0 : 1.0 / 216.0));
    }
  }
  for (int i = 0; i < lat.Q; ++i)
    for (int j = 0; j < lat.Q; ++j)
      if (lat.c[j][0] == -lat.c[i][0] && lat.c[j][1] == -lat.c[i][1] &&
          lat.c[j][2] == -lat.c[i][2])
        lat.opp[i] = j;
  return lat;
}

// ---------------------------------------------------------------- constants
enum { TIME_LINEAR = 0, TIME_TWO_LAYER = 1, TIME_DIFFUSIVE = 2 };
enum { BC_PERIODIC = 0, BC_WALL = 1, BC_VELOCITY_IN = 2, BC_PRESSURE_OUT = 3 };
enum Kind { FLUID = 0, GFC = 1, GFF = 2 };
enum LinkKind { LK_SELF, LK_PULL, LK_BOUNCE, LK_INLET, LK_OUT_NORMAL, LK_OUT_EXTRAP };
enum CellState { CS_OUT, CS_LEAF, CS_SUB, CS_COARSER, CS_SOLID };
constexpr double kM = 2.0;  // m = dx_c / dx_f (Sec. 2.2)

using Coord = std::array<int64_t, 3>;

inline int64_t pack(const Coord& p) {
  // Coordinates are non-negative and below 2^21 here.
  return (p[0] << 42) | (p[1] << 21) | p[2];
}

struct Link {
  int kind = LK_SELF;
  int src = -1;     // element index (same level) for LK_PULL
  int a = -1, b = -1;  // extrapolation sources for LK_OUT_EXTRAP; a: second node x + c_i of an obstacle link
  int face = -1;
  bool obstacle = false;
  double q = 0.5;      // obstacle link: wall at x - q c_i (Bouzidi); 1/2 is half-way bounce-back
  double s = 1.0;      // inlet link: velocity profile factor at the boundary point
};

template <class T>
struct Elem {
  Kind kind = FLUID;
  int layer = 0;
  Coord x{};
  int64_t user = -1;
  std::vector<T> f, fn;  // current post-collision state f*, and the next one
  T F[3] = {T(0.0), T(0.0), T(0.0)};
  std::vector<Link> link;
  bool processed = false;
  int src[4] = {-1, -1, -1, -1};  // GFC: H,K,M,N (3D) or H,E,N,NE (2D) on level L-1
  int sgn[3] = {1, 1, 1};         // GFC: octant of the ghost relative to its parent
  int child[8] = {-1, -1, -1, -1, -1, -1, -1, -1};  // GFF: children on level L+1
};

template <class T>
struct Level {
  int L = 0;
  T omega = T(0.0);
  double uin_scale = 1.0;  // inlet velocity of this level per unit of the coarsest level's
  std::vector<Elem<T>> e;
  std::unordered_map<int64_t, int> at;
  std::unordered_set<int64_t> leaf, sub;
};

// Moments of one element taken from its stored post-collision pdfs.
template <class T>
struct Mom {
  T rho;
  T u[3];
  T S[6];       // xx,yy,zz,xy,yz,xz (3D) or xx,yy,xy (2D)
  T fneq[kQmax];  // pre-collision non-equilibrium part
};

template <class T>
struct Sim {
  Lattice lat;
  int d = 0, Q = 0, mode = TIME_LINEAR;
  // time-step ratio dt_c / dt_f of a level interface: 2 with acoustic scaling
  // (dt proportional to dx), 4 with the diffusive scaling (dt proportional to
  // dx^2) that Sec. 2.2 mentions for the multi-layer scheme
  double mt() const { return mode == TIME_DIFFUSIVE ? 4.0 : kM; }
  // f^neq has an even part in c (first order in the Chapman-Enskog
  // expansion: the viscous stress, proportional to tau dt S) and an odd part
  // (a vector flux, proportional to tau dt^2 / dx: dt^2 / dx (rho d_t u +
  // grad p) from the first-order term, and tau^2 dx dt grad^2 u from the
  // second-order one, which is of the same order when dt ~ dx^2).  Eq.
  // (fneq_scale) carries the even part from one level to the next by the
  // ratio of tau dt.  With acoustic scaling dt / dx is the same on both
  // levels, so the odd part takes the same ratio.  With diffusive scaling its
  // ratio is smaller by (dt_f / dt_c) / (dx_f / dx_c) = 1/2 from coarse to
  // fine (2 from fine to coarse): odd_ratio, the extra factor.
  double odd_ratio(bool to_coarse) const {
    if (mode != TIME_DIFFUSIVE) return 1.0;
    return to_coarse ? mt() / kM : kM / mt();
  }
  // f^neq_i -> even_i + r odd_i, even / odd the halves of f^neq_i +- f^neq_opp(i)
  void odd_rescale(T* fn, double r) const {
    if (r == 1.0) return;
    T out[kQmax];
    for (int i = 0; i < Q; ++i) {
      const T ev = (fn[i] + fn[lat.opp[i]]) / T(2.0), od = (fn[i] - fn[lat.opp[i]]) / T(2.0);
      out[i] = ev + T(r) * od;
    }
    for (int i = 0; i < Q; ++i) fn[i] = out[i];
  }
  int64_t ext0[3] = {1, 1, 1};
  int bc[6] = {0, 0, 0, 0, 0, 0};
  double rho0 = 1.0;
  double uin[3] = {0.0, 0.0, 0.0};
  T uinT[3] = {T(0.0), T(0.0), T(0.0)};  // inlet velocity carried in T (tangent for the dual twin)
  bool outlet_zero_gradient = false;     // outlet extrapolation order 0 instead of 1

  // Inlet velocity profile: 0 uniform, 1 parabolic in the axes tangential to
  // the inlet face, 6 t (1 - t) per axis with t the boundary point's position
  // across the domain (mean 1).  The boundary point of the link i of element x
  // is x - c_i / 2.
  void set_inlet_profile(int profile) {
    for (int li = 0; li < nlev(); ++li)
      for (auto& e : lv[li].e)
        for (int i = 1; i < Q; ++i) {
          Link& lk = e.link[i];
          if (lk.kind != LK_INLET) continue;
          lk.s = 1.0;
          if (profile != 1) continue;
          int nface = -1;
          for (int f = 0; f < 2 * d; ++f)
            if (bc[f] == BC_VELOCITY_IN) nface = f / 2;
          for (int a = 0; a < d; ++a) {
            if (a == nface) continue;
            const double t = (e.x[a] + 0.5 - 0.5 * lat.c[i][a]) / (double)ext(li, a);
            lk.s *= 6.0 * t * (1.0 - t);
          }
        }
  }

  // Wall distance of obstacle links, given per (user element, direction i with
  // x - c_i solid); false if a pair is not an obstacle link or q is outside (0,1].
  bool set_link_q(int64_t n, const int64_t* user, const int* dir, const double* q) {
    for (int64_t k = 0; k < n; ++k) {
      if (user[k] < 0 || user[k] >= (int64_t)upos.size() || dir[k] < 1 || dir[k] >= Q) return false;
      if (!(q[k] > 0.0 && q[k] <= 1.0)) return false;
      auto& e = lv[upos[user[k]].first].e[upos[user[k]].second];
      Link& lk = e.link[dir[k]];
      if (lk.kind != LK_BOUNCE || !lk.obstacle) return false;
      lk.q = q[k];
    }
    return true;
  }
  bool use_force = false;
  T omega_c = T(1.0);
  int n_levels_req = 0;  // 0: the levels the treeIDs span
  int Lmin = 0, Lmax = 0;
  std::vector<Level<T>> lv;
  std::vector<std::pair<int, int>> upos;
  std::string err;

  int nlev() const { return (int)lv.size(); }
  bool periodic(int a) const { return bc[2 * a] == BC_PERIODIC; }
  int64_t ext(int li, int a) const { return a < d ? (ext0[a] << li) : 1; }

  // ------------------------------------------------------------ equilibrium
  // Eq. (feq), c_s^2 = 1/3, with the u.u term subtracted.
  T feq(int i, const T& rho, const T* u) const {
    T cu = T(0.0), uu = T(0.0);
    for (int a = 0; a < d; ++a) {
      cu += T((double)lat.c[i][a]) * u[a];
      uu += u[a] * u[a];
    }
    return T(lat.w[i]) * rho * (T(1.0) + T(3.0) * cu + T(4.5) * cu * cu - T(1.5) * uu);
  }

  // Guo forcing term (the paper has no body force; this is the reading used for
  // the body-force objective): (1 - omega/2) w_i [3 (c_i - u) + 9 (c_i.u) c_i].F
  T guo(int i, const T& omega, const T* u, const T* F) const {
    T cu = T(0.0), cF = T(0.0), uF = T(0.0);
    for (int a = 0; a < d; ++a) {
      cu += T((double)lat.c[i][a]) * u[a];
      cF += T((double)lat.c[i][a]) * F[a];
      uF += u[a] * F[a];
    }
    return (T(1.0) - omega / T(2.0)) * T(lat.w[i]) *
           (T(3.0) * (cF - uF) + T(9.0) * cu * cF);
  }

  // ------------------------------------------------------------ cell lookup
  int cell_state(int li, Coord p, Coord* wrapped, int* faces) const {
    int fc = 0;
    for (int a = 0; a < d; ++a) {
      int64_t n = ext(li, a);
      if (periodic(a)) {
        p[a] = ((p[a] % n) + n) % n;
      } else if (p[a] < 0) {
        fc |= 1 << (2 * a);
      } else if (p[a] >= n) {
        fc |= 1 << (2 * a + 1);
      }
    }
    if (wrapped) *wrapped = p;
    if (faces) *faces = fc;
    if (fc) return CS_OUT;
    int64_t k = pack(p);
    if (lv[li].leaf.count(k)) return CS_LEAF;
    if (lv[li].sub.count(k)) return CS_SUB;
    for (int l2 = li - 1; l2 >= 0; --l2) {
      Coord q = p;
      for (int a = 0; a < d; ++a) q[a] = p[a] >> (li - l2);
      if (lv[l2].leaf.count(pack(q))) return CS_COARSER;
    }
    return CS_SOLID;
  }

  int index_at(int li, const Coord& p) const {
    Coord w;
    int fc;
    int st = cell_state(li, p, &w, &fc);
    if (st == CS_OUT) return -1;
    auto it = lv[li].at.find(pack(w));
    return it == lv[li].at.end() ? -1 : it->second;
  }

  // ------------------------------------------------------------ mesh
  // treeID decoding (Sec. 3.1): level L holds ids off(L) .. off(L+1)-1 with
  // off(L) = (2^{dL}-1)/(2^d-1); the remainder is the z-curve (Morton) index
  // at that level with the x bit lowest.
  bool decode(int64_t t, int* L, Coord* x) const {
    if (t < 0) return false;
    int64_t nch = (int64_t)1 << d;
    int64_t off = 0, cnt = 1;
    int lev = 0;
    while (true) {
      if (t < off + cnt) break;
      off += cnt;
      if (cnt > (INT64_MAX / nch)) return false;
      cnt *= nch;
      ++lev;
      if (lev > 20) return false;
    }
    int64_t m = t - off;
    Coord p{0, 0, 0};
    for (int b = 0; b < lev; ++b)
      for (int a = 0; a < d; ++a) p[a] |= ((m >> (d * b + a)) & 1) << b;
    *L = lev;
    *x = p;
    return true;
  }

  bool fail(const std::string& s) {
    err = s;
    return false;
  }

  bool build(const int64_t* tid, int64_t n) {
    if (n <= 0) return fail("empty mesh");
    std::vector<int> L(n);
    std::vector<Coord> X(n);
    for (int64_t k = 0; k < n; ++k)
      if (!decode(tid[k], &L[k], &X[k])) return fail("invalid treeID");
    Lmin = *std::min_element(L.begin(), L.end());
    Lmax = *std::max_element(L.begin(), L.end());
    // an explicit level count may add finer levels that hold no element yet
    // (an empty refined region): the recursive stepping of Sec. 2.2 still runs
    // through them
    if (n_levels_req > 0) {
      if (n_levels_req < Lmax - Lmin + 1) return fail("n_levels below the levels the treeIDs span");
      Lmax = Lmin + n_levels_req - 1;
    }
    for (int a = 0; a < d; ++a)
      if (ext0[a] < 1 || ext0[a] > ((int64_t)1 << Lmin)) return fail("extent outside the bounding cube");
    lv.assign(Lmax - Lmin + 1, Level<T>());
    for (int li = 0; li < nlev(); ++li) lv[li].L = Lmin + li;
    // relaxation per level, Eq. (fneq_scale): 1/w_f - 1/2 = m (1/w_c - 1/2)
    // (acoustic scaling).  Diffusive scaling keeps the lattice viscosity, so
    // omega is the same on every level: the factor is dx_c^2 dt_f / (dx_f^2 dt_c)
    lv[0].omega = omega_c;
    for (int li = 1; li < nlev(); ++li)
      lv[li].omega = T(1.0) / (T(0.5) + T(kM * kM / mt()) * (T(1.0) / lv[li - 1].omega - T(0.5)));
    for (int li = 0; li < nlev(); ++li) lv[li].uin_scale = std::pow(kM / mt(), li);
    for (int64_t k = 0; k < n; ++k) {
      int li = L[k] - Lmin;
      for (int a = 0; a < d; ++a)
        if (X[k][a] >= ext(li, a)) return fail("element outside the domain box");
      if (!lv[li].leaf.insert(pack(X[k])).second) return fail("duplicate treeID");
    }
    for (int64_t k = 0; k < n; ++k) {
      int li = L[k] - Lmin;
      for (int l2 = li - 1; l2 >= 0; --l2) {
        Coord q = X[k];
        for (int a = 0; a < d; ++a) q[a] >>= (li - l2);
        lv[l2].sub.insert(pack(q));
      }
    }
    for (int li = 0; li < nlev(); ++li)
      for (int64_t k : lv[li].leaf)
        if (lv[li].sub.count(k)) return fail("overlapping elements");
    // fluid elements, kept in the user's order on each level
    upos.resize(n);
    for (int64_t k = 0; k < n; ++k) {
      int li = L[k] - Lmin;
      Elem<T> e;
      e.kind = FLUID;
      e.x = X[k];
      e.user = k;
      upos[k] = {li, (int)lv[li].e.size()};
      lv[li].at[pack(X[k])] = (int)lv[li].e.size();
      lv[li].e.push_back(std::move(e));
    }
    const int nl = mode == TIME_LINEAR ? 2 : 1;
    const int nch = 1 << d;
    // GhostFromFiner: refined cells of level L within nl cells of level-L fluid.
    for (int li = 0; li + 1 < nlev(); ++li) {
      std::unordered_map<int64_t, int> layer;
      std::vector<Coord> order;
      int nfl = (int)lv[li].e.size();
      for (int k = 0; k < nfl; ++k) {
        const Coord x = lv[li].e[k].x;
        for (int oz = (d == 3 ? -nl : 0); oz <= (d == 3 ? nl : 0); ++oz)
          for (int oy = -nl; oy <= nl; ++oy)
            for (int ox = -nl; ox <= nl; ++ox) {
              Coord p{x[0] + ox, x[1] + oy, x[2] + oz};
              Coord w;
              int fc;
              if (cell_state(li, p, &w, &fc) != CS_SUB) continue;
              int dist = std::max(std::abs(ox), std::max(std::abs(oy), std::abs(oz)));
              auto it = layer.find(pack(w));
              if (it == layer.end()) {
                layer[pack(w)] = dist;
                order.push_back(w);
              } else {
                it->second = std::min(it->second, dist);
              }
            }
      }
      for (const Coord& w : order) {
        Elem<T> g;
        g.kind = GFF;
        g.x = w;
        g.layer = layer[pack(w)];
        for (int b = 0; b < nch; ++b) {
          Coord c{2 * w[0] + (b & 1), 2 * w[1] + ((b >> 1) & 1), d == 3 ? 2 * w[2] + ((b >> 2) & 1) : 0};
          auto it = lv[li + 1].at.find(pack(c));
          if (!lv[li + 1].leaf.count(pack(c)) || it == lv[li + 1].at.end())
            return fail("GhostFromFiner child is not a fluid element");
          g.child[b] = it->second;
        }
        lv[li].at[pack(w)] = (int)lv[li].e.size();
        lv[li].e.push_back(std::move(g));
      }
    }
    // GhostFromCoarser: all children of level L-1 fluid parents within R coarse
    // cells of the refined region: two fine layers around the fine fluid
    // (R = 1), four with diffusive scaling (R = 2), Sec. 2.2.
    const int R = mode == TIME_DIFFUSIVE ? 2 : 1;
    for (int li = 1; li < nlev(); ++li) {
      int nparent = (int)lv[li - 1].e.size();
      for (int k = 0; k < nparent; ++k) {
        if (lv[li - 1].e[k].kind != FLUID) continue;
        const Coord P = lv[li - 1].e[k].x;
        bool touches = false;
        for (int oz = (d == 3 ? -R : 0); oz <= (d == 3 ? R : 0) && !touches; ++oz)
          for (int oy = -R; oy <= R && !touches; ++oy)
            for (int ox = -R; ox <= R && !touches; ++ox) {
              Coord p{P[0] + ox, P[1] + oy, P[2] + oz};
              if (cell_state(li - 1, p, nullptr, nullptr) == CS_SUB) touches = true;
            }
        if (!touches) continue;
        for (int b = 0; b < nch; ++b) {
          Elem<T> g;
          g.kind = GFC;
          int bit[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
          g.x = {2 * P[0] + bit[0], 2 * P[1] + bit[1], d == 3 ? 2 * P[2] + bit[2] : 0};
          for (int a = 0; a < 3; ++a) g.sgn[a] = (a < d && bit[a]) ? 1 : -1;
          // layer: the Chebyshev distance to the nearest fine fluid (or more
          // refined) cell, the outermost layer (2, or 4) also for farther ghosts
          const int nlay = 2 * R;
          g.layer = nlay;
          for (int oz = (d == 3 ? -(nlay - 1) : 0); oz <= (d == 3 ? nlay - 1 : 0); ++oz)
            for (int oy = -(nlay - 1); oy <= nlay - 1; ++oy)
              for (int ox = -(nlay - 1); ox <= nlay - 1; ++ox) {
                const int dist = std::max(std::abs(ox), std::max(std::abs(oy), std::abs(oz)));
                if (dist == 0 || dist >= g.layer) continue;
                int st = cell_state(li, Coord{g.x[0] + ox, g.x[1] + oy, g.x[2] + oz}, nullptr, nullptr);
                if (st == CS_LEAF || st == CS_SUB) g.layer = dist;
              }
          // sources on level L-1 (Sec. 2.2): the parent H and, in the octant of
          // the ghost, K=(1,1,0), M=(1,0,1), N=(0,1,1) in 3D; in 2D the square
          // H=(0,0), E=(1,0), N=(0,1), NE=(1,1).
          int off3[4][3] = {{0, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
          int off2[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {1, 1, 0}};
          for (int s = 0; s < 4; ++s) {
            const int* o = d == 3 ? off3[s] : off2[s];
            Coord q{P[0] + g.sgn[0] * o[0], P[1] + g.sgn[1] * o[1], d == 3 ? P[2] + g.sgn[2] * o[2] : 0};
            int idx = index_at(li - 1, q);
            if (idx < 0 || lv[li - 1].e[idx].kind == GFC)
              return fail("GhostFromCoarser source is neither fluid nor GhostFromFiner");
            g.src[s] = idx;
          }
          Coord w;
          int fc;
          cell_state(li, g.x, &w, &fc);
          if (lv[li].at.count(pack(w))) return fail("GhostFromCoarser collides with another element");
          lv[li].at[pack(w)] = (int)lv[li].e.size();
          lv[li].e.push_back(std::move(g));
        }
      }
    }
    // which elements the stream-collide step advances
    for (int li = 0; li < nlev(); ++li)
      for (auto& e : lv[li].e)
        e.processed = e.kind == FLUID || (e.kind == GFC && e.layer == 1 && mode == TIME_TWO_LAYER) ||
                      (e.kind == GFC && e.layer <= 3 && mode == TIME_DIFFUSIVE) ||
                      (e.kind == GFF && e.layer == 1 && mode == TIME_LINEAR);
    // pull links (Sec. 2.1 streaming, Sec. 2.3 boundaries)
    for (int li = 0; li < nlev(); ++li) {
      for (auto& e : lv[li].e) {
        e.f.assign(Q, T(0.0));
        e.fn.assign(Q, T(0.0));
        e.link.assign(Q, Link());
        if (!e.processed) continue;
        for (int i = 1; i < Q; ++i) {
          Coord p{e.x[0] - lat.c[i][0], e.x[1] - lat.c[i][1], e.x[2] - lat.c[i][2]};
          Coord w;
          int fc;
          int st = cell_state(li, p, &w, &fc);
          Link lk;
          if (st == CS_OUT) {
            if (e.kind != FLUID) return fail("ghost element next to the domain boundary");
            bool wall = false, inl = false;
            int nout = 0, oface = -1;
            for (int f = 0; f < 2 * d; ++f) {
              if (!(fc & (1 << f))) continue;
              if (bc[f] == BC_WALL) wall = true;
              if (bc[f] == BC_VELOCITY_IN) inl = true;
              if (bc[f] == BC_PRESSURE_OUT) {
                ++nout;
                oface = f;
              }
            }
            if (wall) {
              lk.kind = LK_BOUNCE;
            } else if (inl) {
              lk.kind = LK_INLET;
            } else {
              if (nout != 1) return fail("outlet corner without wall");
              lk.face = oface;
              int a = oface / 2, sg = (oface & 1) ? 1 : -1;
              int nrm[3] = {0, 0, 0};
              nrm[a] = sg;
              bool normal = true;
              for (int b = 0; b < 3; ++b)
                if (lat.c[i][b] != -nrm[b]) normal = false;
              if (normal) {
                lk.kind = LK_OUT_NORMAL;
              } else {
                lk.kind = LK_OUT_EXTRAP;
                Coord pa{p[0] - nrm[0], p[1] - nrm[1], p[2] - nrm[2]};
                Coord pb{p[0] - 2 * nrm[0], p[1] - 2 * nrm[1], p[2] - 2 * nrm[2]};
                lk.a = index_at(li, pa);
                lk.b = index_at(li, pb);
                if (lk.a < 0 || lk.b < 0 || lv[li].e[lk.a].kind != FLUID || lv[li].e[lk.b].kind != FLUID)
                  return fail("outlet extrapolation source missing");
              }
            }
          } else {
            auto it = lv[li].at.find(pack(w));
            if (it != lv[li].at.end()) {
              lk.kind = LK_PULL;
              lk.src = it->second;
            } else if (st == CS_SOLID) {
              if (e.kind != FLUID) return fail("ghost element next to a solid");
              lk.kind = LK_BOUNCE;
              lk.obstacle = true;
              // second node of the interpolated bounce-back: the element
              // behind x, away from the wall (any element of this level)
              lk.a = index_at(li, Coord{e.x[0] + lat.c[i][0], e.x[1] + lat.c[i][1], e.x[2] + lat.c[i][2]});
            } else {
              return fail("neighbour on another level has no ghost element");
            }
          }
          e.link[i] = lk;
        }
      }
    }
    // start from rest equilibrium everywhere (ghosts are overwritten by the
    // first fill)
    for (auto& l : lv)
      for (auto& e : l.e)
        for (int i = 0; i < Q; ++i) e.f[i] = T(lat.w[i] * rho0);
    return true;
  }

  // ------------------------------------------------------------ moments
  // rho = sum f*, rho u = sum c f* - F/2 (post-collision storage with Guo
  // forcing), pre-collision f^neq = (f* - f^eq - F_i)/(1 - omega), and the
  // strain rate S_ab = -(3 omega / 2 rho) sum_i c_ia c_ib f^neq_i.
  void moments(const Elem<T>& e, const T& omega, Mom<T>* m) const {
    T rho = T(0.0);
    T j[3] = {T(0.0), T(0.0), T(0.0)};
    for (int i = 0; i < Q; ++i) {
      rho += e.f[i];
      for (int a = 0; a < d; ++a) j[a] += T((double)lat.c[i][a]) * e.f[i];
    }
    m->rho = rho;
    for (int a = 0; a < 3; ++a) m->u[a] = a < d ? (j[a] - e.F[a] / T(2.0)) / rho : T(0.0);
    for (int i = 0; i < Q; ++i)
      m->fneq[i] = (e.f[i] - feq(i, rho, m->u) - guo(i, omega, m->u, e.F)) / (T(1.0) - omega);
    const int pa[6] = {0, 1, 2, 0, 1, 0}, pb[6] = {0, 1, 2, 1, 2, 2};
    const int pa2[3] = {0, 1, 0}, pb2[3] = {0, 1, 1};
    int ns = d == 3 ? 6 : 3;
    for (int s = 0; s < 6; ++s) m->S[s] = T(0.0);
    for (int s = 0; s < ns; ++s) {
      int a = d == 3 ? pa[s] : pa2[s], b = d == 3 ? pb[s] : pb2[s];
      T acc = T(0.0);
      for (int i = 0; i < Q; ++i) acc += T((double)(lat.c[i][a] * lat.c[i][b])) * m->fneq[i];
      m->S[s] = -(T(3.0) * omega / (T(2.0) * rho)) * acc;
    }
  }

  // ------------------------------------------------------------ BGK step
  // Eq. (bgk) in pull form: f_i(x, t+1) = f*_i(x - c_i, t), then
  // f* = f - omega (f - f^eq) + F_i.
  T pull(const Level<T>& l, const Elem<T>& e, int i) const {
    const Link& lk = e.link[i];
    int ib = lat.opp[i];
    switch (lk.kind) {
      case LK_SELF:
        return e.f[i];
      case LK_PULL:
        return l.e[lk.src].f[i];
      case LK_BOUNCE: {
        if (!lk.obstacle) return e.f[ib];
        // linearly interpolated bounce-back (Bouzidi, Sec. 2.3): the pdf
        // leaving toward the wall at x - q c_i returns as
        //   q <  1/2: 2q f*_ib(x) + (1 - 2q) f*_ib(x + c_i)
        //   q >= 1/2: f*_ib(x) / (2q) + (2q - 1)/(2q) f*_i(x)
        // (q = 1/2 is half-way bounce-back; without a node behind x the link
        // falls back to it)
        const double q = lk.q;
        if (q < 0.5) {
          if (lk.a < 0) return e.f[ib];
          return T(2.0 * q) * e.f[ib] + T(1.0 - 2.0 * q) * l.e[lk.a].f[ib];
        }
        return T(1.0 / (2.0 * q)) * e.f[ib] + T((2.0 * q - 1.0) / (2.0 * q)) * e.f[i];
      }
      case LK_INLET: {
        // velocity bounce-back (Ladd): f_i = f*_ib + 2 w_i rho0 (c_i.U) / c_s^2,
        // U = u_in times the profile factor at the boundary point
        T cu = T(0.0);
        for (int a = 0; a < d; ++a) cu += T((double)lat.c[i][a]) * uinT[a] * T(l.uin_scale);
        return e.f[ib] + T(6.0 * lat.w[i] * rho0 * lk.s) * cu;
      }
      case LK_OUT_NORMAL: {
        // pressure-corrected outlet along the normal: f^eq_i(rho0, u) + f^neq_ib.
        // The incoming value is a pre-collision pdf, so f^neq_ib is the
        // pre-collision non-equilibrium part of the opposite pdf (the same
        // quantity the interpolation of Sec. 2.2 works with), recovered from
        // the stored post-collision values by moments().
        Mom<T> m;
        moments(e, l.omega, &m);
        return feq(i, T(rho0), m.u) + m.fneq[ib];
      }
      case LK_OUT_EXTRAP:
        // extrapolation of the missing outside element along -n: linear
        // (Sec. 2.3) or, as an option, zero-gradient
        if (outlet_zero_gradient) return l.e[lk.a].f[i];
        return T(2.0) * l.e[lk.a].f[i] - l.e[lk.b].f[i];
    }
    return e.f[i];
  }

  // The element loops below touch one element each (reading others' stored
  // pdfs only), so they may run on several threads with the same result.
  void stream_collide(int li) {
    Level<T>& l = lv[li];
    const T omega = l.omega;
    const int64_t ne = (int64_t)l.e.size();
#pragma omp parallel for schedule(static) if (ne >= kParMin)
    for (int64_t k = 0; k < ne; ++k) {
      Elem<T>& e = l.e[k];
      if (!e.processed) continue;
      T fin[kQmax];
      for (int i = 0; i < Q; ++i) fin[i] = pull(l, e, i);
      T rho = T(0.0);
      T j[3] = {T(0.0), T(0.0), T(0.0)};
      for (int i = 0; i < Q; ++i) {
        rho += fin[i];
        for (int a = 0; a < d; ++a) j[a] += T((double)lat.c[i][a]) * fin[i];
      }
      T u[3] = {T(0.0), T(0.0), T(0.0)};
      for (int a = 0; a < d; ++a) u[a] = (j[a] + e.F[a] / T(2.0)) / rho;
      for (int i = 0; i < Q; ++i)
        e.fn[i] = fin[i] - omega * (fin[i] - feq(i, rho, u)) + guo(i, omega, u, e.F);
    }
#pragma omp parallel for schedule(static) if (ne >= kParMin)
    for (int64_t k = 0; k < ne; ++k)
      if (l.e[k].processed) l.e[k].f.swap(l.e[k].fn);
  }

  // ------------------------------------------------------------ GhostFromFiner
  // Coarse ghost from its 2^d children (Sec. 2.2, interpolation steps 1-5 with
  // the children as sources).  The ghost sits at the children's centroid, so
  // the linear interpolation of density and f^neq is their plain mean.  The
  // velocity is interpolated quadratically: for a quadratic field the
  // children's mean exceeds the centre value by (1/32) lap u (children at
  // +-1/4 coarse cell), and lap u_a = 2 d_b S_ab - d_a S_bb follows from the
  // children's strain rates, whose derivatives are differences across the
  // children's cube of side 1/2.  f^neq is rescaled to the coarse level by
  // m omega_f / omega_c (inverse of the GFC rescale); then f = f^eq + f^neq is
  // stored as a post-collision value.
  void fill_gff(int li) {
    Level<T>& lc = lv[li];
    const Level<T>& lf = lv[li + 1];
    const int nch = 1 << d;
    const int64_t ng = (int64_t)lc.e.size();
#pragma omp parallel for schedule(static) if (ng >= kParMin)
    for (int64_t k = 0; k < ng; ++k) {
      Elem<T>& g = lc.e[k];
      if (g.kind != GFF) continue;
      Mom<T> mk[8];
      for (int b = 0; b < nch; ++b) moments(lf.e[g.child[b]], lf.omega, &mk[b]);
      T rho = T(0.0);
      T u[3] = {T(0.0), T(0.0), T(0.0)};
      T fneq[kQmax];
      for (int i = 0; i < Q; ++i) fneq[i] = T(0.0);
      for (int b = 0; b < nch; ++b) {
        rho += mk[b].rho;
        for (int a = 0; a < d; ++a) u[a] += mk[b].u[a];
        for (int i = 0; i < Q; ++i) fneq[i] += mk[b].fneq[i];
      }
      rho = rho / T((double)nch);
      for (int a = 0; a < d; ++a) u[a] = u[a] / T((double)nch);
      if (mode == TIME_DIFFUSIVE) {
        // to coarse lattice units: u_c = (dt_c / dt_f) / (dx_c / dx_f) u_f, and
        // the density deviation (a pressure) scales with the square of that
        const double us = mt() / kM;
        rho = T(rho0) + T(us * us) * (rho - T(rho0));
        for (int a = 0; a < d; ++a) u[a] = T(us) * u[a];
      }
      // strain rate of every child in coarse lattice units: S_c = (dt_c/dt_f) S_f
      auto S_c = [&](int b, int a1, int a2) {
        int idx;
        if (a1 == a2) idx = a1;
        else if (d == 2) idx = 2;
        else {
          int lo = std::min(a1, a2), hi = std::max(a1, a2);
          idx = lo == 0 ? (hi == 1 ? 3 : 5) : 4;  // xy, xz, yz
        }
        return T(mt()) * mk[b].S[idx];
      };
      // d/dx_c of a child quantity: (mean over children on the + side minus
      // mean on the - side) / (1/2)
      auto deriv = [&](int c, auto&& phi) {
        T plus = T(0.0), minus = T(0.0);
        for (int b = 0; b < nch; ++b) {
          if ((b >> c) & 1) plus += phi(b); else minus += phi(b);
        }
        return (plus - minus) / T((double)(nch / 2)) / T(0.5);
      };
      for (int a = 0; a < d; ++a) {
        T lap = T(0.0);
        for (int c = 0; c < d; ++c) {
          lap += T(2.0) * deriv(c, [&](int b) { return S_c(b, a, c); });
          lap -= deriv(a, [&](int b) { return S_c(b, c, c); });
        }
        u[a] = u[a] - lap / T(32.0);
      }
      const T scale = T(mt()) * lf.omega / lc.omega;
      odd_rescale(fneq, odd_ratio(true));
      for (int i = 0; i < Q; ++i) {
        T fn = scale * fneq[i] / T((double)nch);
        g.f[i] = feq(i, rho, u) + (T(1.0) - lc.omega) * fn;
      }
    }
  }

  // ------------------------------------------------------------ GhostFromCoarser
  // Source moments of the coarse level, one record per coarse element.
  std::vector<Mom<T>> level_moments(int li) const {
    const Level<T>& l = lv[li];
    std::vector<Mom<T>> out(l.e.size());
    const int64_t ne = (int64_t)l.e.size();
#pragma omp parallel for schedule(static) if (ne >= kParMin)
    for (int64_t k = 0; k < ne; ++k)
      if (l.e[k].kind != GFC) moments(l.e[k], l.omega, &out[k]);
    return out;
  }

  void fill_gfc(int li, const std::vector<Mom<T>>& q0, const std::vector<Mom<T>>* q1);

  // The ops of advance() one at a time, for a driver that interleaves its own
  // steps (the halo exchange of a partitioned run): source moments at t (A)
  // and t+1 (B) are kept per level between calls.
  std::vector<std::vector<Mom<T>>> op_qa, op_qb;
  bool run_op(int op, int li) {
    if (li < 0 || li >= nlev()) return false;
    op_qa.resize(nlev());
    op_qb.resize(nlev());
    const bool finer = li + 1 < nlev();
    switch (op) {
      case 0:  // GhostFromFiner of level li
        if (!finer) return false;
        fill_gff(li);
        return true;
      case 1:  // source moments of level li at t
        op_qa[li] = level_moments(li);
        return true;
      case 2:  // GhostFromCoarser of level li+1 from the moments at t
        if (!finer || op_qa[li].size() != lv[li].e.size()) return false;
        fill_gfc(li + 1, op_qa[li], nullptr);
        return true;
      case 3:  // stream + collide of level li
        stream_collide(li);
        return true;
      case 4:  // source moments of level li at t+1
        op_qb[li] = level_moments(li);
        return true;
      case 5:  // GhostFromCoarser of level li+1 from the mean of t and t+1
        if (!finer || op_qa[li].size() != lv[li].e.size() || op_qb[li].size() != lv[li].e.size()) return false;
        fill_gfc(li + 1, op_qa[li], &op_qb[li]);
        return true;
    }
    return false;
  }

  // ------------------------------------------------------------ driver
  // Recursive level time stepping (Sec. 2.2): one step on level L is two on
  // level L+1 (acoustic scaling); GFF is filled before GFC at the synchronous
  // time.  LINEAR mode also refills GFC before the second fine substep from the
  // mean of the coarse source moments at t and t+1 (linear interpolation in
  // time); TWO_LAYER mode instead lets the fine kernel advance the inner ghost
  // layer (the paper's scheme).
  void advance(int li) {
    std::vector<Mom<T>> qt;
    if (li + 1 < nlev()) {
      fill_gff(li);
      qt = level_moments(li);
      fill_gfc(li + 1, qt, nullptr);
    }
    stream_collide(li);
    if (li + 1 < nlev() && mode == TIME_DIFFUSIVE) {
      // four fine substeps on the four ghost layers filled above
      for (int k = 0; k < 4; ++k) advance(li + 1);
      return;
    }
    if (li + 1 < nlev()) {
      advance(li + 1);
      if (mode == TIME_LINEAR) {
        std::vector<Mom<T>> qt1 = level_moments(li);
        fill_gfc(li + 1, qt, &qt1);
      }
      advance(li + 1);
    }
  }

  void fill_ghosts() {
    for (int li = 0; li + 1 < nlev(); ++li) {
      fill_gff(li);
      std::vector<Mom<T>> q = level_moments(li);
      fill_gfc(li + 1, q, nullptr);
    }
  }
};

// Compact quadratic velocity (Sec. 2.2).  Inputs in the global frame: the four
// sources' velocity and strain rate (coarse lattice units) and the octant signs
// of the ghost relative to the parent H.  The problem is reflected into the
// octant's local frame, where the sources sit at H(0,0,0), K(1,1,0), M(1,0,1),
// N(0,1,1) and the ghost at (1/4,1/4,1/4); the 18 quadratic coefficients come
// from the strain-rate differences (Eqs. compact_3D_s), then the 12 constant
// and linear ones from the source velocities (Eqs. compact_3D_u).
template <class T>
void compact_velocity_3d(const int s[3], const T u[4][3], const T S[4][6], T out[3]) {
  T ul[4][3], Sl[4][6];
  for (int k = 0; k < 4; ++k) {
    for (int a = 0; a < 3; ++a) ul[k][a] = T((double)s[a]) * u[k][a];
    Sl[k][0] = S[k][0];
    Sl[k][1] = S[k][1];
    Sl[k][2] = S[k][2];
    Sl[k][3] = T((double)(s[0] * s[1])) * S[k][3];
    Sl[k][4] = T((double)(s[1] * s[2])) * S[k][4];
    Sl[k][5] = T((double)(s[0] * s[2])) * S[k][5];
  }
  enum { XX = 0, YY = 1, ZZ = 2, XY = 3, YZ = 4, XZ = 5 };
  // 2 dPhi/dx = -Phi(H) + Phi(K) + Phi(M) - Phi(N), and likewise for y, z
  auto two_dx = [&](int c) { return -Sl[0][c] + Sl[1][c] + Sl[2][c] - Sl[3][c]; };
  auto two_dy = [&](int c) { return -Sl[0][c] + Sl[1][c] - Sl[2][c] + Sl[3][c]; };
  auto two_dz = [&](int c) { return -Sl[0][c] - Sl[1][c] + Sl[2][c] + Sl[3][c]; };
  // Eqs. (compact_3D_s), solved for the quadratic coefficients
  T axx = two_dx(XX) / T(4.0), axy = two_dy(XX) / T(2.0), axz = two_dz(XX) / T(2.0);
  T bxy = two_dx(YY) / T(2.0), byy = two_dy(YY) / T(4.0), byz = two_dz(YY) / T(2.0);
  T cxz = two_dx(ZZ) / T(2.0), cyz = two_dy(ZZ) / T(2.0), czz = two_dz(ZZ) / T(4.0);
  T bxx = (two_dx(XY) - axy) / T(2.0);   // a_xy + 2 b_xx = 2 dSxy/dx
  T ayy = (two_dy(XY) - bxy) / T(2.0);   // 2 a_yy + b_xy = 2 dSxy/dy
  T cyy = (two_dy(YZ) - byz) / T(2.0);   // b_yz + 2 c_yy = 2 dSyz/dy
  T bzz = (two_dz(YZ) - cyz) / T(2.0);   // 2 b_zz + c_yz = 2 dSyz/dz
  T cxx = (two_dx(XZ) - axz) / T(2.0);   // a_xz + 2 c_xx = 2 dSxz/dx
  T azz = (two_dz(XZ) - cxz) / T(2.0);   // 2 a_zz + c_xz = 2 dSxz/dz
  // a_yz + b_xz = 2 dSxy/dz, b_xz + c_xy = 2 dSyz/dx, a_yz + c_xy = 2 dSxz/dy
  T r1 = two_dz(XY), r2 = two_dx(YZ), r3 = two_dy(XZ);
  T half = (r1 + r2 + r3) / T(2.0);
  T ayz = half - r2, bxz = half - r3, cxy = half - r1;
  T q[3][6] = {{axx, ayy, azz, axy, ayz, axz},
               {bxx, byy, bzz, bxy, byz, bxz},
               {cxx, cyy, czz, cxy, cyz, cxz}};
  const double P[4][3] = {{0, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
  auto quad = [&](int comp, double x, double y, double z) {
    const T* c = q[comp];
    return c[0] * T(x * x) + c[1] * T(y * y) + c[2] * T(z * z) + c[3] * T(x * y) + c[4] * T(y * z) +
           c[5] * T(x * z);
  };
  for (int comp = 0; comp < 3; ++comp) {
    // Eqs. (compact_3D_u): u(H) = a0; u(K) = a0+ax+ay+quad(K); ...
    T a0 = ul[0][comp];
    T rK = ul[1][comp] - a0 - quad(comp, P[1][0], P[1][1], P[1][2]);  // = ax + ay
    T rM = ul[2][comp] - a0 - quad(comp, P[2][0], P[2][1], P[2][2]);  // = ax + az
    T rN = ul[3][comp] - a0 - quad(comp, P[3][0], P[3][1], P[3][2]);  // = ay + az
    T ax = (rK + rM - rN) / T(2.0);
    T ay = (rK - rM + rN) / T(2.0);
    T az = (-rK + rM + rN) / T(2.0);
    T val = a0 + (ax + ay + az) * T(0.25) + quad(comp, 0.25, 0.25, 0.25);
    out[comp] = T((double)s[comp]) * val;
  }
}

// 2D counterpart on the unit square H(0,0), E(1,0), N(0,1), NE(1,1) with the
// ghost at (1/4,1/4).  The quadratic coefficients come from the strain-rate
// differences as in 3D; the constant and linear coefficients are the
// least-squares plane through the four residual velocities (four equations,
// three unknowns per component).
template <class T>
void compact_velocity_2d(const int s[3], const T u[4][3], const T S[4][6], T out[3]) {
  T ul[4][2], Sl[4][3];
  for (int k = 0; k < 4; ++k) {
    for (int a = 0; a < 2; ++a) ul[k][a] = T((double)s[a]) * u[k][a];
    Sl[k][0] = S[k][0];
    Sl[k][1] = S[k][1];
    Sl[k][2] = T((double)(s[0] * s[1])) * S[k][2];
  }
  auto two_dx = [&](int c) { return -Sl[0][c] + Sl[1][c] - Sl[2][c] + Sl[3][c]; };
  auto two_dy = [&](int c) { return -Sl[0][c] - Sl[1][c] + Sl[2][c] + Sl[3][c]; };
  T axx = two_dx(0) / T(4.0), axy = two_dy(0) / T(2.0);
  T bxy = two_dx(1) / T(2.0), byy = two_dy(1) / T(4.0);
  T bxx = (two_dx(2) - axy) / T(2.0);
  T ayy = (two_dy(2) - bxy) / T(2.0);
  T q[2][3] = {{axx, ayy, axy}, {bxx, byy, bxy}};
  const double P[4][2] = {{0, 0}, {1, 0}, {0, 1}, {1, 1}};
  for (int comp = 0; comp < 2; ++comp) {
    T r[4];
    for (int k = 0; k < 4; ++k) {
      double x = P[k][0], y = P[k][1];
      r[k] = ul[k][comp] - (q[comp][0] * T(x * x) + q[comp][1] * T(y * y) + q[comp][2] * T(x * y));
    }
    // normal equations of the plane fit over the square's corners
    T ax = (-r[0] + r[1] - r[2] + r[3]) / T(2.0);
    T ay = (-r[0] - r[1] + r[2] + r[3]) / T(2.0);
    T a0 = (r[0] + r[1] + r[2] + r[3]) / T(4.0) - (ax + ay) / T(2.0);
    T val = a0 + (ax + ay) * T(0.25) +
            (q[comp][0] + q[comp][1] + q[comp][2]) * T(1.0 / 16.0);
    out[comp] = T((double)s[comp]) * val;
  }
  out[2] = T(0.0);
}

// Interpolation steps 1-5 of Sec. 2.2 for every GhostFromCoarser of level li.
// q1 (LINEAR mode, second fine substep) averages the source moments at t and
// t+1 before interpolating.
template <class T>
void Sim<T>::fill_gfc(int li, const std::vector<Mom<T>>& q0, const std::vector<Mom<T>>* q1) {
  Level<T>& lf = lv[li];
  const Level<T>& lc = lv[li - 1];
  const int ns = d == 3 ? 6 : 3;
  // linear (barycentric / bilinear) weights of the ghost position
  const double w3[4] = {5.0 / 8.0, 1.0 / 8.0, 1.0 / 8.0, 1.0 / 8.0};
  const double w2[4] = {9.0 / 16.0, 3.0 / 16.0, 3.0 / 16.0, 1.0 / 16.0};
  const double* lw = d == 3 ? w3 : w2;
  const int64_t ng = (int64_t)lf.e.size();
#pragma omp parallel for schedule(static) if (ng >= kParMin)
  for (int64_t kg = 0; kg < ng; ++kg) {
    Elem<T>& g = lf.e[kg];
    if (g.kind != GFC) continue;
    // step 1: moments at the sources
    Mom<T> m[4];
    for (int k = 0; k < 4; ++k) {
      m[k] = q0[g.src[k]];
      if (q1) {
        const Mom<T>& b = (*q1)[g.src[k]];
        m[k].rho = (m[k].rho + b.rho) / T(2.0);
        for (int a = 0; a < 3; ++a) m[k].u[a] = (m[k].u[a] + b.u[a]) / T(2.0);
        for (int s = 0; s < 6; ++s) m[k].S[s] = (m[k].S[s] + b.S[s]) / T(2.0);
        for (int i = 0; i < Q; ++i) m[k].fneq[i] = (m[k].fneq[i] + b.fneq[i]) / T(2.0);
      }
    }
    // step 2: velocity quadratically, density and f^neq linearly
    T us[4][3], Ss[4][6];
    for (int k = 0; k < 4; ++k) {
      for (int a = 0; a < 3; ++a) us[k][a] = m[k].u[a];
      for (int s = 0; s < 6; ++s) Ss[k][s] = s < ns ? m[k].S[s] : T(0.0);
    }
    T u[3];
    if (d == 3)
      compact_velocity_3d<T>(g.sgn, us, Ss, u);
    else
      compact_velocity_2d<T>(g.sgn, us, Ss, u);
    T rho = T(0.0);
    for (int k = 0; k < 4; ++k) rho += T(lw[k]) * m[k].rho;
    if (mode == TIME_DIFFUSIVE) {
      // to fine lattice units (inverse of the GhostFromFiner conversion)
      const double us = kM / mt();
      rho = T(rho0) + T(us * us) * (rho - T(rho0));
      for (int a = 0; a < d; ++a) u[a] = T(us) * u[a];
    }
    // step 4: rescale f^neq, omega_c f^neq_c / m = omega_f f^neq_f (m the
    // time-step ratio)
    const T scale = lc.omega / (T(mt()) * lf.omega);
    T fn[kQmax];
    for (int i = 0; i < Q; ++i) {
      fn[i] = T(0.0);
      for (int k = 0; k < 4; ++k) fn[i] += T(lw[k]) * m[k].fneq[i];
    }
    odd_rescale(fn, odd_ratio(false));
    for (int i = 0; i < Q; ++i) {
      // steps 3 and 5: f = f^eq + f^neq, stored post-collision
      g.f[i] = feq(i, rho, u) + (T(1.0) - lf.omega) * (scale * fn[i]);
    }
  }
}

template <class T>
struct Handle {
  Sim<T> sim;
};

template <class T>
Sim<T>* create_sim(int stencil, int time_mode, const int* extent, const int* bc, double omega_c,
                   double omega_dot, double rho0, const double* u_in, const double* u_in_dot, int use_force,
                   const int64_t* tree_ids, int64_t n, int n_levels, char* err, int errlen) {
  auto* s = new Sim<T>();
  auto bail = [&](const char* m) -> Sim<T>* {
    if (err && errlen > 0) snprintf(err, errlen, "%s", m);
    delete s;
    return nullptr;
  };
  if (stencil != 9 && stencil != 19 && stencil != 27) return bail("stencil must be 9, 19 or 27");
  if (time_mode != TIME_LINEAR && time_mode != TIME_TWO_LAYER && time_mode != TIME_DIFFUSIVE) return bail("bad time mode");
  s->lat = make_lattice(stencil);
  s->d = s->lat.d;
  s->Q = s->lat.Q;
  s->mode = time_mode;
  for (int a = 0; a < 3; ++a) s->ext0[a] = a < s->d ? extent[a] : 1;
  for (int f = 0; f < 6; ++f) s->bc[f] = f < 2 * s->d ? bc[f] : BC_PERIODIC;
  for (int a = 0; a < s->d; ++a)
    if ((s->bc[2 * a] == BC_PERIODIC) != (s->bc[2 * a + 1] == BC_PERIODIC))
      return bail("periodic must be set on both faces of an axis");
  if (!(omega_c > 0.0 && omega_c < 2.0)) return bail("omega must lie in (0,2)");
  s->omega_c = T(omega_c);
  if constexpr (std::is_same<T, Dual>::value) s->omega_c = Dual(omega_c, omega_dot);
  s->rho0 = rho0;
  for (int a = 0; a < 3; ++a) {
    s->uin[a] = u_in ? u_in[a] : 0.0;
    s->uinT[a] = T(s->uin[a]);
    if constexpr (std::is_same<T, Dual>::value) s->uinT[a] = Dual(s->uin[a], u_in_dot ? u_in_dot[a] : 0.0);
  }
  s->use_force = use_force != 0;
  if (n_levels < 0 || n_levels > 16) return bail("n_levels must lie in 0..16");
  s->n_levels_req = n_levels;
  if (!s->build(tree_ids, n)) return bail(s->err.c_str());
  for (auto& l : s->lv)
    if (std::fabs(1.0 - value_of(l.omega)) < 1e-3) return bail("omega too close to 1 on some level");
  return s;
}

// f*(0) = f^eq(rho,u) + (1-omega) f^neq(S) + df with the initial
// non-equilibrium part f^neq_i = -(w_i rho / (c_s^2 omega)) Q_i : S,
// Q_i = c_i c_i - c_s^2 I (Sec. 4.1; prefactor such that the strain-rate
// equation returns S).
template <class T>
int init_sim(Sim<T>* s, const double* rho, const double* u, const double* S, const double* df) {
  const int d = s->d, Q = s->Q, ns = d == 3 ? 6 : 3;
  const int pa[6] = {0, 1, 2, 0, 1, 0}, pb[6] = {0, 1, 2, 1, 2, 2};
  const int pa2[3] = {0, 1, 0}, pb2[3] = {0, 1, 1};
  for (size_t k = 0; k < s->upos.size(); ++k) {
    auto& l = s->lv[s->upos[k].first];
    auto& e = l.e[s->upos[k].second];
    T r = T(rho[k]);
    T uu[3] = {T(0.0), T(0.0), T(0.0)};
    for (int a = 0; a < d; ++a) uu[a] = T(u[k * d + a]);
    for (int i = 0; i < Q; ++i) {
      T fneq = T(0.0);
      if (S) {
        T qs = T(0.0), tr = T(0.0);
        for (int c = 0; c < ns; ++c) {
          int a = d == 3 ? pa[c] : pa2[c], b = d == 3 ? pb[c] : pb2[c];
          double sym = a == b ? 1.0 : 2.0;
          qs += T(sym * s->lat.c[i][a] * s->lat.c[i][b]) * T(S[k * ns + c]);
          if (a == b) tr += T(S[k * ns + c]);
        }
        fneq = -(T(3.0 * s->lat.w[i]) * r / l.omega) * (qs - tr / T(3.0));
      }
      e.f[i] = s->feq(i, r, uu) + (T(1.0) - l.omega) * fneq;
      if (df) e.f[i] += T(df[k * Q + i]);
    }
  }
  return 0;
}

template <class T>
void reduce_sim(const Sim<T>* s, T out[8]) {
  for (int k = 0; k < 8; ++k) out[k] = T(0.0);
  const int d = s->d;
  for (int li = 0; li < s->nlev(); ++li) {
    const auto& l = s->lv[li];
    const double vol = std::ldexp(1.0, -d * li);
    const double fscale = std::ldexp(1.0, (d - 1) * (s->nlev() - 1 - li));
    // diffusive scaling: density deviation, momentum and kinetic energy in the
    // coarsest level's lattice units, forces in the finest level's (the level's
    // velocity unit is (mt/2)^li of the coarsest's; a force unit scales with
    // dx^(d+1) / dt^2)
    const bool dif = s->mode == TIME_DIFFUSIVE;
    const double us = dif ? std::pow(s->mt() / kM, li) : 1.0;
    const double fs = dif ? std::ldexp(1.0, (d - 3) * (s->nlev() - 1 - li)) : fscale;
    for (const auto& e : l.e) {
      if (e.kind != FLUID) continue;
      Mom<T> m;
      s->moments(e, l.omega, &m);
      if (dif) {
        out[0] += T(vol) * (T(s->rho0) + T(us * us) * (m.rho - T(s->rho0)));
        T uu = T(0.0);
        for (int a = 0; a < d; ++a) {
          out[1 + a] += T(vol * us) * m.rho * m.u[a];
          uu += m.u[a] * m.u[a];
        }
        out[7] += T(0.5 * vol * us * us) * m.rho * uu;
      } else {
        out[0] += T(vol) * m.rho;
        T uu = T(0.0);
        for (int a = 0; a < d; ++a) {
          out[1 + a] += T(vol) * m.rho * m.u[a];
          uu += m.u[a] * m.u[a];
        }
        out[7] += T(0.5 * vol) * m.rho * uu;
      }
      // momentum exchange on obstacle links (Sec. 2.3): the pdf f*_ib(x_b)
      // leaves toward the body and f_i(x_b) (the bounce-back value of the next
      // step) returns, so the link carries c_ib (f*_ib + f_i) to the body; with
      // half-way bounce-back that is 2 c_ib f*_ib.
      for (int i = 1; i < s->Q; ++i) {
        if (e.link[i].kind != LK_BOUNCE || !e.link[i].obstacle) continue;
        int ib = s->lat.opp[i];
        const T back = s->pull(l, e, i);
        for (int a = 0; a < d; ++a)
          out[4 + a] += T(fs * s->lat.c[ib][a]) * (e.f[ib] + back);
      }
    }
  }
}

}  // namespace

// ======================================================================= C API
extern "C" {

void* orc_create(int stencil, int time_mode, const int* extent, const int* bc, double omega_c,
                 double rho0, const double* u_in, int use_force, const int64_t* tree_ids, int64_t n,
                 int n_levels, char* err, int errlen) {
  return create_sim<double>(stencil, time_mode, extent, bc, omega_c, 0.0, rho0, u_in, nullptr, use_force,
                            tree_ids, n, n_levels, err, errlen);
}

void orc_destroy(void* h) { delete static_cast<Sim<double>*>(h); }

// Threads of the element loops (stream-collide, ghost fills, source moments);
// n <= 0 keeps the OpenMP default.  Returns the count now in use (1 without
// OpenMP).  Every element is computed by the same arithmetic whatever the
// count, so results do not depend on it.
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

// per level: level, fluid, GFC, GFF, GFC layer-1, GFF layer-1  (6 int64 each)
int orc_counts(void* h, int64_t* out, int cap) {
  auto* s = static_cast<Sim<double>*>(h);
  int n = 0;
  for (auto& l : s->lv) {
    if (n >= cap) break;
    int64_t c[6] = {l.L, 0, 0, 0, 0, 0};
    for (auto& e : l.e) {
      c[1 + e.kind]++;
      if (e.kind == GFC && e.layer == 1) c[4]++;
      if (e.kind == GFF && e.layer == 1) c[5]++;
    }
    std::memcpy(out + 6 * n, c, sizeof(c));
    ++n;
  }
  return n;
}

double orc_level_omega(void* h, int li) {
  auto* s = static_cast<Sim<double>*>(h);
  return li >= 0 && li < s->nlev() ? s->lv[li].omega : -1.0;
}

int orc_init(void* h, const double* rho, const double* u, const double* S, const double* df) {
  return init_sim(static_cast<Sim<double>*>(h), rho, u, S, df);
}

// Outlet extrapolation: 0 = linear (Sec. 2.3), 1 = zero-gradient.
int orc_set_outlet(void* h, int mode) {
  static_cast<Sim<double>*>(h)->outlet_zero_gradient = mode == 1;
  return mode == 0 || mode == 1 ? 0 : -1;
}

int orc_set_inlet_profile(void* h, int profile) {
  if (profile != 0 && profile != 1) return -1;
  static_cast<Sim<double>*>(h)->set_inlet_profile(profile);
  return 0;
}

int orc_set_link_q(void* h, int64_t n, const int64_t* user, const int* dir, const double* q) {
  return static_cast<Sim<double>*>(h)->set_link_q(n, user, dir, q) ? 0 : -1;
}

int orc_set_force(void* h, const double* F) {
  auto* s = static_cast<Sim<double>*>(h);
  for (size_t k = 0; k < s->upos.size(); ++k) {
    auto& e = s->lv[s->upos[k].first].e[s->upos[k].second];
    for (int a = 0; a < s->d; ++a) e.F[a] = F[k * s->d + a];
  }
  return 0;
}

int orc_step(void* h, int64_t n) {
  auto* s = static_cast<Sim<double>*>(h);
  for (int64_t k = 0; k < n; ++k) s->advance(0);
  return 0;
}

int orc_fill_ghosts(void* h) {
  static_cast<Sim<double>*>(h)->fill_ghosts();
  return 0;
}

// One op of the recursive step (0 GhostFromFiner of level li, 1 / 4 source
// moments of level li at t / t+1, 2 / 5 GhostFromCoarser of level li+1 from
// the moments at t / their mean with t+1, 3 stream-collide of level li), for a
// driver that runs the ops in advance()'s order with its own steps in
// between.  Returns -1 for an op that does not apply.
int orc_op(void* h, int op, int li) { return static_cast<Sim<double>*>(h)->run_op(op, li) ? 0 : -1; }

int orc_nlev(void* h) { return static_cast<Sim<double>*>(h)->nlev(); }

// rho[n], u[n][d], S[n][d(d+1)/2] (each element in its own level's lattice
// units), user order
int orc_moments(void* h, double* rho, double* u, double* S) {
  auto* s = static_cast<Sim<double>*>(h);
  const int ns = s->d == 3 ? 6 : 3;
  for (size_t k = 0; k < s->upos.size(); ++k) {
    auto& l = s->lv[s->upos[k].first];
    Mom<double> m;
    s->moments(l.e[s->upos[k].second], l.omega, &m);
    if (rho) rho[k] = m.rho;
    if (u)
      for (int a = 0; a < s->d; ++a) u[k * s->d + a] = m.u[a];
    if (S)
      for (int c = 0; c < ns; ++c) S[k * ns + c] = m.S[c];
  }
  return 0;
}

// fluid post-collision pdfs f*[n][Q], user order
int orc_get_f(void* h, double* f) {
  auto* s = static_cast<Sim<double>*>(h);
  for (size_t k = 0; k < s->upos.size(); ++k) {
    auto& e = s->lv[s->upos[k].first].e[s->upos[k].second];
    for (int i = 0; i < s->Q; ++i) f[k * s->Q + i] = e.f[i];
  }
  return 0;
}

int orc_set_f(void* h, const double* f) {
  auto* s = static_cast<Sim<double>*>(h);
  for (size_t k = 0; k < s->upos.size(); ++k) {
    auto& e = s->lv[s->upos[k].first].e[s->upos[k].second];
    for (int i = 0; i < s->Q; ++i) e.f[i] = f[k * s->Q + i];
  }
  return 0;
}

int64_t orc_ghost_count(void* h) {
  auto* s = static_cast<Sim<double>*>(h);
  int64_t n = 0;
  for (auto& l : s->lv)
    for (auto& e : l.e)
      if (e.kind != FLUID) ++n;
  return n;
}

// ghosts: info[n][6] = level, kind (1 GFC, 2 GFF), layer, x, y, z ; f[n][Q]
int orc_ghosts(void* h, int64_t* info, double* f) {
  auto* s = static_cast<Sim<double>*>(h);
  int64_t n = 0;
  for (auto& l : s->lv)
    for (auto& e : l.e) {
      if (e.kind == FLUID) continue;
      int64_t r[6] = {l.L, e.kind, e.layer, e.x[0], e.x[1], e.x[2]};
      std::memcpy(info + 6 * n, r, sizeof(r));
      for (int i = 0; i < s->Q; ++i) f[n * s->Q + i] = e.f[i];
      ++n;
    }
  return 0;
}

// mass, momentum[3], obstacle force[3] (finest-level lattice units), kinetic
// energy; volumes relative to a coarsest-level element
int orc_reduce(void* h, double* out) {
  reduce_sim(static_cast<Sim<double>*>(h), out);
  return 0;
}

// compact quadratic velocity of one ghost: d = 2 or 3, s = octant signs,
// u4[4][d], S4[4][d(d+1)/2] in the global frame, out[d]
int orc_compact_velocity(int d, const int* s, const double* u4, const double* S4, double* out) {
  double u[4][3] = {}, S[4][6] = {}, o[3] = {};
  int sg[3] = {1, 1, 1};
  const int ns = d == 3 ? 6 : 3;
  for (int a = 0; a < d; ++a) sg[a] = s[a];
  for (int k = 0; k < 4; ++k) {
    for (int a = 0; a < d; ++a) u[k][a] = u4[k * d + a];
    for (int c = 0; c < ns; ++c) S[k][c] = S4[k * ns + c];
  }
  if (d == 3)
    compact_velocity_3d<double>(sg, u, S, o);
  else if (d == 2)
    compact_velocity_2d<double>(sg, u, S, o);
  else
    return -1;
  for (int a = 0; a < d; ++a) out[a] = o[a];
  return 0;
}

// ---------------------------------------------------------- dual-number twin
// Same oracle with every value carrying a tangent: omega_c has tangent
// omega_dot, the inlet velocity u_in_dot and the body force field F_dot, so
// every output's tangent is its directional derivative along
// (F_dot, omega_dot, u_in_dot).
void* orc_dual_create(int stencil, int time_mode, const int* extent, const int* bc, double omega_c,
                      double omega_dot, double rho0, const double* u_in, const double* u_in_dot,
                      int use_force, const int64_t* tree_ids, int64_t n, int n_levels, char* err,
                      int errlen) {
  return create_sim<Dual>(stencil, time_mode, extent, bc, omega_c, omega_dot, rho0, u_in, u_in_dot,
                          use_force, tree_ids, n, n_levels, err, errlen);
}

void orc_dual_destroy(void* h) { delete static_cast<Sim<Dual>*>(h); }

int orc_dual_init(void* h, const double* rho, const double* u, const double* S, const double* df) {
  return init_sim(static_cast<Sim<Dual>*>(h), rho, u, S, df);
}

int orc_dual_set_outlet(void* h, int mode) {
  static_cast<Sim<Dual>*>(h)->outlet_zero_gradient = mode == 1;
  return mode == 0 || mode == 1 ? 0 : -1;
}

int orc_dual_set_inlet_profile(void* h, int profile) {
  if (profile != 0 && profile != 1) return -1;
  static_cast<Sim<Dual>*>(h)->set_inlet_profile(profile);
  return 0;
}

int orc_dual_set_link_q(void* h, int64_t n, const int64_t* user, const int* dir, const double* q) {
  return static_cast<Sim<Dual>*>(h)->set_link_q(n, user, dir, q) ? 0 : -1;
}

int orc_dual_set_force(void* h, const double* F, const double* F_dot) {
  auto* s = static_cast<Sim<Dual>*>(h);
  for (size_t k = 0; k < s->upos.size(); ++k) {
    auto& e = s->lv[s->upos[k].first].e[s->upos[k].second];
    for (int a = 0; a < s->d; ++a)
      e.F[a] = Dual(F[k * s->d + a], F_dot ? F_dot[k * s->d + a] : 0.0);
  }
  return 0;
}

// set the fluid pdfs f*[n][Q] (caller order) with tangents f_dot (NULL: zero)
int orc_dual_set_f(void* h, const double* f, const double* f_dot) {
  auto* s = static_cast<Sim<Dual>*>(h);
  for (size_t k = 0; k < s->upos.size(); ++k) {
    auto& e = s->lv[s->upos[k].first].e[s->upos[k].second];
    for (int i = 0; i < s->Q; ++i) e.f[i] = Dual(f[k * s->Q + i], f_dot ? f_dot[k * s->Q + i] : 0.0);
  }
  return 0;
}

int orc_dual_step(void* h, int64_t n) {
  auto* s = static_cast<Sim<Dual>*>(h);
  for (int64_t k = 0; k < n; ++k) s->advance(0);
  return 0;
}

int orc_dual_reduce(void* h, double* out, double* out_dot) {
  Dual o[8];
  reduce_sim(static_cast<Sim<Dual>*>(h), o);
  for (int k = 0; k < 8; ++k) {
    out[k] = o[k].v;
    out_dot[k] = o[k].d;
  }
  return 0;
}

}  // extern "C"
