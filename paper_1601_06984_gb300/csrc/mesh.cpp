// Host mesh builder: treeID list -> level-wise, z-curve ordered element arrays,
// ghost elements, pull neighbour lists and boundary tables (Sec. 2.2, 2.3, 3.1, 3.2
// of arXiv:1601.06984).  Runs once per mesh, off the hot path; O(n log n) with
// dense per-level lookup grids over each level's bounding box.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>
#include <unordered_map>

#include "lbm_internal.h"

#ifdef _OPENMP
#include <omp.h>
#include <parallel/algorithm>
#define LBM_SORT __gnu_parallel::sort
#else
#define LBM_SORT std::sort
#endif

namespace lbm {
namespace {

// Discrete velocities in the order documented in lbm.h.
struct Dirs {
  int Q = 9, d = 2;
  int c[kQmax][3] = {};
};

Dirs make_dirs(int Q) {
  Dirs r;
  r.Q = Q;
  r.d = Q == 9 ? 2 : 3;
  double w[kQmax];
  host_lattice(Q, r.c, w);
  return r;
}

inline int64_t pad_up(int64_t n) { return (n + kPad - 1) / kPad * kPad; }

// z-curve key of integer coordinates (x bit lowest)
inline uint64_t zkey(const int64_t* x, int d, int bits) {
  uint64_t k = 0;
  for (int b = 0; b < bits; ++b)
    for (int a = 0; a < d; ++a) k |= (uint64_t)((x[a] >> b) & 1) << (d * b + a);
  return k;
}

bool decode_tid(int64_t t, int d, int* L, int64_t x[3]) {
  if (t < 0) return false;
  const int64_t nch = (int64_t)1 << d;
  int64_t off = 0, cnt = 1;
  int lev = 0;
  while (t >= off + cnt) {
    off += cnt;
    cnt *= nch;
    if (++lev > (d == 3 ? 20 : 30)) return false;
  }
  const uint64_t m = (uint64_t)(t - off);
  x[0] = x[1] = x[2] = 0;
  for (int b = 0; b < lev; ++b)
    for (int a = 0; a < d; ++a) x[a] |= (int64_t)((m >> (d * b + a)) & 1) << b;
  *L = lev;
  return true;
}

struct Grid {
  int64_t lo[3] = {0, 0, 0}, n[3] = {1, 1, 1};
  std::vector<int32_t> g;  // -1 nothing, -2 subdivided (no ghost), >= 0 local element index
  int64_t at(const int64_t* p) const {
    int64_t o = 0;
    for (int a = 2; a >= 0; --a) {
      int64_t q = p[a] - lo[a];
      if (q < 0 || q >= n[a]) return -1;
      o = o * n[a] + q;
    }
    return o;
  }
};

constexpr int32_t G_NONE = -1, G_SUB = -2;

struct Ghost {
  uint64_t key;
  int64_t x[3];
  int layer;
  uint8_t oct;
};

struct Builder {
  int d = 2, Q = 9, mode = 0;
  int64_t ext0[3] = {1, 1, 1};
  int bc[6] = {0, 0, 0, 0, 0, 0};
  Dirs dr;
  int Lmin = 0, Lmax = 0, nlev = 1;
  std::vector<Grid> grid;
  std::vector<std::vector<uint8_t>> kind;  // per level, local index -> K_*
  std::string err;

  bool periodic(int a) const { return bc[2 * a] == LBM_BC_PERIODIC; }
  int64_t ext(int li, int a) const { return a < d ? (ext0[a] << li) : 1; }

  // wrap periodic axes; returns the bitmask of crossed (non-periodic) faces
  int wrap(int li, int64_t* p) const {
    int fc = 0;
    for (int a = 0; a < d; ++a) {
      const int64_t n = ext(li, a);
      if (periodic(a)) {
        p[a] = ((p[a] % n) + n) % n;
      } else if (p[a] < 0) {
        fc |= 1 << (2 * a);
      } else if (p[a] >= n) {
        fc |= 1 << (2 * a + 1);
      }
    }
    return fc;
  }

  int32_t value(int li, const int64_t* p) const {
    int64_t o = grid[li].at(p);
    return o < 0 ? G_NONE : grid[li].g[o];
  }

  // Is the (wrapped, in-box) cell p of level li covered by a coarser fluid element?
  bool covered_by_coarser(int li, const int64_t* p) const {
    for (int l2 = li - 1; l2 >= 0; --l2) {
      int64_t q[3] = {p[0] >> (li - l2), p[1] >> (li - l2), p[2] >> (li - l2)};
      int32_t v = value(l2, q);
      if (v == G_SUB) return false;
      if (v >= 0) {
        uint8_t k = kind[l2][v];
        if (k == K_FLUID) return true;
        if (k == K_GFF) return false;
        // a GhostFromCoarser is itself covered by an even coarser element
      }
    }
    return false;
  }

  bool fail(const char* m) {
    if (err.empty()) err = m;
    return false;
  }
};

}  // namespace

lbm_status build_host_mesh(const int64_t* tid, const int8_t* levels, int64_t n, const lbm_params& p,
                           HostMesh* out, std::string* msg) {
  Builder B;
  auto bad = [&](lbm_status s, const std::string& m) {
    *msg = m;
    return s;
  };
  if (!tid || n <= 0) return bad(LBM_ERR_ARG, "empty mesh");
  if (p.stencil != 9 && p.stencil != 19 && p.stencil != 27) return bad(LBM_ERR_ARG, "stencil must be 9, 19 or 27");
  if (p.time_mode != LBM_TIME_LINEAR && p.time_mode != LBM_TIME_TWO_LAYER && p.time_mode != LBM_TIME_DIFFUSIVE)
    return bad(LBM_ERR_ARG, "bad time mode");
  if (p.inlet_profile != LBM_INLET_UNIFORM && p.inlet_profile != LBM_INLET_PARABOLIC)
    return bad(LBM_ERR_ARG, "bad inlet profile");
  if (p.bouzidi != 0 && p.bouzidi != 1) return bad(LBM_ERR_ARG, "bouzidi must be 0 or 1");
  if (!(p.omega_coarse > 0.0 && p.omega_coarse < 2.0)) return bad(LBM_ERR_ARG, "omega must lie in (0,2)");
  if (!(p.rho0 > 0.0)) return bad(LBM_ERR_ARG, "rho0 must be positive");
  B.Q = p.stencil;
  B.d = p.stencil == 9 ? 2 : 3;
  B.mode = p.time_mode;
  B.dr = make_dirs(B.Q);
  const int d = B.d, Q = B.Q;
  for (int a = 0; a < 3; ++a) B.ext0[a] = a < d ? p.extent[a] : 1;
  for (int f = 0; f < 6; ++f) B.bc[f] = f < 2 * d ? p.bc[f] : LBM_BC_PERIODIC;
  for (int f = 0; f < 2 * d; ++f)
    if (B.bc[f] < 0 || B.bc[f] > 3) return bad(LBM_ERR_ARG, "bad boundary kind");
  for (int a = 0; a < d; ++a)
    if ((B.bc[2 * a] == LBM_BC_PERIODIC) != (B.bc[2 * a + 1] == LBM_BC_PERIODIC))
      return bad(LBM_ERR_ARG, "periodic must be set on both faces of an axis");

  // ---- decode (Sec. 3.1)
  std::vector<int8_t> L(n);
  std::vector<int64_t> X(3 * n);
  int bad_id = 0, bad_lvl = 0;
#pragma omp parallel for schedule(static) reduction(| : bad_id, bad_lvl)
  for (int64_t k = 0; k < n; ++k) {
    int lev = 0;
    if (!decode_tid(tid[k], d, &lev, &X[3 * k])) {
      bad_id = 1;
      continue;
    }
    L[k] = (int8_t)lev;
    if (levels && levels[k] != lev) bad_lvl = 1;
  }
  if (bad_id) return bad(LBM_ERR_MESH, "invalid treeID");
  if (bad_lvl) return bad(LBM_ERR_MESH, "level does not match treeID");
  B.Lmin = *std::min_element(L.begin(), L.end());
  B.Lmax = *std::max_element(L.begin(), L.end());
  B.nlev = B.Lmax - B.Lmin + 1;
  if (B.nlev > 16) return bad(LBM_ERR_MESH, "more than 16 levels");
  // an explicit level count may add finer levels with no element yet (an
  // empty refined region); the driver still steps through them
  if (p.n_levels < 0 || p.n_levels > 16) return bad(LBM_ERR_ARG, "n_levels must lie in 0..16");
  if (p.n_levels > 0) {
    if (p.n_levels < B.nlev) return bad(LBM_ERR_ARG, "n_levels below the levels the treeIDs span");
    B.nlev = p.n_levels;
    B.Lmax = B.Lmin + B.nlev - 1;
  }
  for (int a = 0; a < d; ++a)
    if (B.ext0[a] < 1 || B.ext0[a] > ((int64_t)1 << B.Lmin))
      return bad(LBM_ERR_ARG, "extent outside the bounding cube");
  const int nlev = B.nlev;
  int outside = 0;
#pragma omp parallel for schedule(static) reduction(| : outside)
  for (int64_t k = 0; k < n; ++k)
    for (int a = 0; a < d; ++a)
      if (X[3 * k + a] >= B.ext(L[k] - B.Lmin, a)) outside = 1;
  if (outside) return bad(LBM_ERR_MESH, "element outside the domain box");

  // ---- per level z-curve sorted fluid lists (Sec. 3.2)
  std::vector<std::vector<std::pair<uint64_t, int64_t>>> fl(nlev);
  {
    std::vector<int64_t> cnt(nlev, 0);
    for (int64_t k = 0; k < n; ++k) cnt[L[k] - B.Lmin]++;
    for (int li = 0; li < nlev; ++li) fl[li].reserve(cnt[li]);
    for (int64_t k = 0; k < n; ++k) {
      int li = L[k] - B.Lmin;
      fl[li].push_back({zkey(&X[3 * k], d, B.Lmin + li), k});
    }
    for (int li = 0; li < nlev; ++li) {
      LBM_SORT(fl[li].begin(), fl[li].end());
      for (size_t j = 1; j < fl[li].size(); ++j)
        if (fl[li][j].first == fl[li][j - 1].first) return bad(LBM_ERR_MESH, "duplicate treeID");
    }
  }

  // ---- interior bricks.  A brick is an aligned block of 64 same-level fluid
  // elements (4^3 in 3D, 8^2 in 2D), i.e. one run of z-curve keys sharing
  // key >> 6.  A complete brick is interior when every brick its elements pull
  // from (the face and edge neighbours the stencil reaches) is complete too:
  // all its links are plain pulls between fluid elements of one level, and the
  // source of link i at local position l is brick slot t plus local position
  // l', a table common to all bricks.  A complete brick with some neighbour
  // brick missing is a boundary brick: its links through the missing slots
  // take the neighbour list instead.  The level's fluid list becomes interior
  // bricks, boundary bricks, the rest; everything keeps z-curve order within
  // its part (so GhostFromFiner children stay contiguous).
  const int bshift = d == 3 ? 2 : 3, bside = 1 << bshift;
  constexpr int64_t kMissingPos = -1;  // neighbour brick not complete (slot value below)
  std::vector<std::vector<std::array<int64_t, 27>>> brick_nbpos(nlev);  // per brick: slot -> new position
  std::vector<int64_t> n_interior(nlev, 0), n_boundary(nlev, 0);
  {
    // brick offsets the stencil needs: s_a in {0, -c_a}, not all zero
    bool need[27] = {};
    for (int i = 1; i < Q; ++i)
      for (int m = 1; m < (1 << d); ++m) {
        int s3[3] = {0, 0, 0};
        bool ok = true;
        for (int a = 0; a < d; ++a)
          if (m >> a & 1) {
            if (B.dr.c[i][a] == 0) ok = false;
            s3[a] = -B.dr.c[i][a];
          }
        if (ok) need[(s3[0] + 1) + 3 * (s3[1] + 1) + 9 * (s3[2] + 1)] = true;
      }
    for (int li = 0; li < nlev; ++li) {
      auto& f = fl[li];
      const int64_t nf = (int64_t)f.size();
      std::vector<int64_t> cstart;  // original start of each complete brick
      std::unordered_map<uint64_t, int64_t> cidx;
      for (int64_t j = 0; j + 63 < nf;) {
        if ((f[j].first & 63) == 0 && f[j + 63].first == f[j].first + 63) {
          cidx.emplace(f[j].first >> 6, (int64_t)cstart.size());
          cstart.push_back(j);
          j += 64;
        } else {
          ++j;
        }
      }
      const int64_t nc = (int64_t)cstart.size();
      int64_t nbx[3];
      for (int a = 0; a < 3; ++a) nbx[a] = a < d ? (B.ext(li, a) + bside - 1) >> bshift : 1;
      std::vector<std::array<int64_t, 27>> nbc(nc);
      std::vector<uint8_t> interior(nc, 0);
#pragma omp parallel for schedule(static)
      for (int64_t b = 0; b < nc; ++b) {
        const int64_t* x0 = &X[3 * f[cstart[b]].second];
        int64_t bc[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) bc[a] = x0[a] >> bshift;
        bool all = true;
        for (int t = 0; t < 27; ++t) {
          nbc[b][t] = b;
          if (!need[t]) continue;
          const int sx[3] = {t % 3 - 1, t / 3 % 3 - 1, t / 9 - 1};
          int64_t q[3] = {0, 0, 0};
          bool ok = true;
          for (int a = 0; a < d && ok; ++a) {
            q[a] = bc[a] + sx[a];
            if (q[a] < 0 || q[a] >= nbx[a]) {
              // across the domain edge: only a periodic axis whose extent is a
              // whole number of bricks keeps the brick structure
              if (!B.periodic(a) || (B.ext(li, a) & (bside - 1)) != 0) ok = false;
              else q[a] = (q[a] + nbx[a]) % nbx[a];
            }
          }
          auto it = ok ? cidx.find(zkey(q, d, B.Lmin + li - bshift)) : cidx.end();
          if (it == cidx.end()) {
            nbc[b][t] = kMissingPos;
            all = false;
          } else {
            nbc[b][t] = it->second;
          }
        }
        interior[b] = all;
      }
      // new order: interior bricks, boundary bricks, then the rest; new position
      // of every complete brick
      std::vector<int64_t> cnew(nc);
      std::vector<std::pair<uint64_t, int64_t>> g;
      g.reserve(nf);
      int64_t nint = 0, nbnd = 0;
      for (int pass = 0; pass < 2; ++pass)
        for (int64_t b = 0; b < nc; ++b)
          if ((bool)interior[b] == (pass == 0)) {
            cnew[b] = (int64_t)g.size();
            (pass == 0 ? nint : nbnd) += 1;
            g.insert(g.end(), f.begin() + cstart[b], f.begin() + cstart[b] + 64);
          }
      {
        int64_t b = 0;
        for (int64_t j = 0; j < nf; ++j) {
          while (b < nc && cstart[b] + 64 <= j) ++b;
          const bool in_brick = b < nc && cstart[b] <= j;
          if (!in_brick) g.push_back(f[j]);
        }
      }
      f.swap(g);
      n_interior[li] = nint;
      n_boundary[li] = nbnd;
      // rows in the new brick order (interior first, then boundary)
      std::vector<int64_t> order(nc);
      for (int64_t b = 0; b < nc; ++b) order[cnew[b] / 64] = b;
      auto& bn = brick_nbpos[li];
      bn.resize(nc);
      for (int64_t k = 0; k < nc; ++k)
        for (int t = 0; t < 27; ++t) {
          const int64_t src = nbc[order[k]][t];
          bn[k][t] = src == kMissingPos ? kMissingPos : cnew[src];
        }
    }
  }

  // ---- bounding boxes and dense lookup grids
  B.grid.resize(nlev);
  B.kind.resize(nlev);
  {
    std::vector<std::array<int64_t, 6>> bb(nlev);
    for (int li = 0; li < nlev; ++li) bb[li] = {INT64_MAX, INT64_MAX, INT64_MAX, INT64_MIN, INT64_MIN, INT64_MIN};
    for (int li = 0; li < nlev; ++li) {
      int64_t lo[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, hi[3] = {INT64_MIN, INT64_MIN, INT64_MIN};
      for (auto& e : fl[li])
        for (int a = 0; a < d; ++a) {
          lo[a] = std::min(lo[a], X[3 * e.second + a]);
          hi[a] = std::max(hi[a], X[3 * e.second + a]);
        }
      for (int a = 0; a < d; ++a) {
        bb[li][a] = lo[a];
        bb[li][3 + a] = hi[a];
      }
    }
    for (int li = nlev - 2; li >= 0; --li)
      for (int a = 0; a < d; ++a)
        if (bb[li + 1][3 + a] != INT64_MIN) {
          bb[li][a] = std::min(bb[li][a], bb[li + 1][a] >> 1);
          bb[li][3 + a] = std::max(bb[li][3 + a], bb[li + 1][3 + a] >> 1);
        }
    const int64_t margin = 4;
    for (int li = 0; li < nlev; ++li) {
      Grid& G = B.grid[li];
      int64_t vol = 1;
      for (int a = 0; a < 3; ++a) {
        if (a >= d) {
          G.lo[a] = 0;
          G.n[a] = 1;
          continue;
        }
        if (bb[li][3 + a] == INT64_MIN) {  // a level with no element: an empty grid
          G.lo[a] = 0;
          G.n[a] = 1;
          continue;
        }
        int64_t lo = bb[li][a] - margin, hi = bb[li][3 + a] + margin + 1;
        const int64_t e = B.ext(li, a);
        if (B.periodic(a) && (lo < 0 || hi > e)) {
          lo = 0;
          hi = e;
        }
        lo = std::max<int64_t>(lo, 0);
        hi = std::min<int64_t>(hi, e);
        G.lo[a] = lo;
        G.n[a] = std::max<int64_t>(hi - lo, 1);
        vol *= G.n[a];
      }
      if (vol > ((int64_t)1 << 31)) return bad(LBM_ERR_MESH, "level bounding box too large for a dense lookup grid");
      G.g.assign(vol, G_NONE);
    }
  }
  for (int li = 0; li < nlev; ++li) {
    Grid& G = B.grid[li];
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < (int64_t)fl[li].size(); ++r) G.g[G.at(&X[3 * fl[li][r].second])] = (int32_t)r;
  }
  // subdivided cells: parents of fluid or subdivided cells of the next finer level
  for (int li = nlev - 2; li >= 0; --li) {
    const Grid& Gf = B.grid[li + 1];
    Grid& Gc = B.grid[li];
    int64_t c[3];
    for (c[2] = 0; c[2] < Gf.n[2]; ++c[2])
      for (c[1] = 0; c[1] < Gf.n[1]; ++c[1])
        for (c[0] = 0; c[0] < Gf.n[0]; ++c[0]) {
          int32_t v = Gf.g[(c[2] * Gf.n[1] + c[1]) * Gf.n[0] + c[0]];
          if (v == G_NONE) continue;
          int64_t q[3] = {(c[0] + Gf.lo[0]) >> 1, (c[1] + Gf.lo[1]) >> 1, d == 3 ? (c[2] + Gf.lo[2]) >> 1 : 0};
          int64_t o = Gc.at(q);
          if (o < 0) return bad(LBM_ERR_INTERNAL, "parent outside the coarse lookup grid");
          if (Gc.g[o] >= 0) return bad(LBM_ERR_MESH, "overlapping elements");
          Gc.g[o] = G_SUB;
        }
  }
  for (int li = 0; li < nlev; ++li) B.kind[li].assign(fl[li].size(), K_FLUID);

  // ---- GhostFromFiner: subdivided cells within nl cells of level fluid (nl = 2 in LINEAR)
  const int nl = B.mode == LBM_TIME_LINEAR ? 2 : 1;
  const int zr = d == 3 ? 1 : 0;
  std::vector<std::vector<Ghost>> gff(nlev), gfc(nlev);
  for (int li = 0; li + 1 < nlev; ++li) {
    const Grid& G = B.grid[li];
    const int64_t nz = G.n[2], ny = G.n[1], nx = G.n[0];
    std::vector<std::vector<Ghost>> part;
#pragma omp parallel
    {
#ifdef _OPENMP
      const int nt = omp_get_num_threads(), tid_ = omp_get_thread_num();
#else
      const int nt = 1, tid_ = 0;
#endif
#pragma omp single
      part.resize(nt);
      std::vector<Ghost> mine;
#pragma omp for schedule(static)
      for (int64_t s = 0; s < nz * ny; ++s) {
        const int64_t cz = s / ny, cy = s % ny;
        for (int64_t cx = 0; cx < nx; ++cx) {
          if (G.g[(cz * ny + cy) * nx + cx] != G_SUB) continue;
          const int64_t x0[3] = {cx + G.lo[0], cy + G.lo[1], cz + G.lo[2]};
          int best = 99;
          for (int oz = -nl * zr; oz <= nl * zr; ++oz)
            for (int oy = -nl; oy <= nl; ++oy)
              for (int ox = -nl; ox <= nl; ++ox) {
                int dist = std::max(std::abs(ox), std::max(std::abs(oy), std::abs(oz)));
                if (dist == 0 || dist >= best) continue;
                int64_t q[3] = {x0[0] + ox, x0[1] + oy, x0[2] + oz};
                if (B.wrap(li, q)) continue;
                if (B.value(li, q) >= 0) best = dist;
              }
          if (best <= nl) {
            Ghost g;
            for (int a = 0; a < 3; ++a) g.x[a] = x0[a];
            g.key = zkey(g.x, d, B.Lmin + li);
            g.layer = best;
            g.oct = 0;
            mine.push_back(g);
          }
        }
      }
#pragma omp critical
      part[tid_].swap(mine);
    }
    for (auto& v : part) gff[li].insert(gff[li].end(), v.begin(), v.end());
    // inner layer first, each layer z-curve sorted
    LBM_SORT(gff[li].begin(), gff[li].end(), [](const Ghost& a, const Ghost& b) {
      return a.layer != b.layer ? a.layer < b.layer : a.key < b.key;
    });
  }

  // ---- GhostFromCoarser: all children of level L-1 fluid within R coarse cells
  // of a subdivided cell: two fine layers (R = 1), or four with diffusive
  // scaling (R = 2), whose four substeps per coarse step eat one layer each
  const int R = B.mode == LBM_TIME_DIFFUSIVE ? 2 : 1;
  const int nlay = 2 * R;
  for (int li = 1; li < nlev; ++li) {
    const auto& parents = fl[li - 1];
    const int64_t np = (int64_t)parents.size();
    std::vector<uint8_t> touch(np, 0);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < np; ++r) {
      const int64_t* P = &X[3 * parents[r].second];
      for (int oz = -R * zr; oz <= R * zr && !touch[r]; ++oz)
        for (int oy = -R; oy <= R && !touch[r]; ++oy)
          for (int ox = -R; ox <= R; ++ox) {
            int64_t q[3] = {P[0] + ox, P[1] + oy, P[2] + oz};
            if (B.wrap(li - 1, q)) continue;
            if (B.value(li - 1, q) == G_SUB) {
              touch[r] = 1;
              break;
            }
          }
    }
    const int nch = 1 << d;
    for (int64_t r = 0; r < np; ++r) {
      if (!touch[r]) continue;
      const int64_t* P = &X[3 * parents[r].second];
      for (int b = 0; b < nch; ++b) {
        Ghost g;
        g.x[0] = 2 * P[0] + (b & 1);
        g.x[1] = 2 * P[1] + ((b >> 1) & 1);
        g.x[2] = d == 3 ? 2 * P[2] + ((b >> 2) & 1) : 0;
        g.oct = (uint8_t)b;
        g.key = zkey(g.x, d, B.Lmin + li);
        g.layer = nlay;
        gfc[li].push_back(g);
      }
    }
    // layer: the Chebyshev distance to the nearest fluid or subdivided cell of
    // this level, nlay for farther ghosts too
    const int sr = nlay - 1;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < (int64_t)gfc[li].size(); ++k) {
      Ghost& g = gfc[li][k];
      for (int oz = -sr * zr; oz <= sr * zr; ++oz)
        for (int oy = -sr; oy <= sr; ++oy)
          for (int ox = -sr; ox <= sr; ++ox) {
            const int dist = std::max(std::abs(ox), std::max(std::abs(oy), std::abs(oz)));
            if (dist == 0 || dist >= g.layer) continue;
            int64_t q[3] = {g.x[0] + ox, g.x[1] + oy, g.x[2] + oz};
            if (B.wrap(li, q)) continue;
            int32_t v = B.value(li, q);
            if (v >= 0 || v == G_SUB) g.layer = dist;
          }
    }
  }

  // ---- level layout [GFC | fluid | GFF inner | GFF outer], padded segments
  HostMesh& M = *out;
  M = HostMesh();
  M.d = d;
  M.Q = Q;
  M.nS = d == 3 ? 6 : 3;
  M.Lmin = B.Lmin;
  M.Lmax = B.Lmax;
  M.n_user = n;
  M.lv.resize(nlev);
  int64_t base = 0;
  for (int li = 0; li < nlev; ++li) {
    HostLevel& H = M.lv[li];
    H.L = B.Lmin + li;
    H.nC = (int64_t)gfc[li].size();
    H.nF = (int64_t)fl[li].size();
    H.nG1 = 0;
    for (auto& g : gff[li]) H.nG1 += g.layer == 1;
    H.nG2 = (int64_t)gff[li].size() - H.nG1;
    H.oC = 0;
    H.oF = pad_up(H.nC);
    H.oG1 = H.oF + pad_up(H.nF);
    H.oG2 = H.oG1 + pad_up(H.nG1);
    H.N = H.oG2 + pad_up(H.nG2);
    H.base = base;
    base += H.N;
  }
  M.Ntot = base;
  if (M.Ntot >= (int64_t)NB_INDEX) return bad(LBM_ERR_MESH, "too many elements for 30-bit neighbour indices");
  // interior bricks: global first-element index of each neighbour brick, and
  // the (slot, local position) table of every link
  {
    int64_t rows = 0;
    for (int li = 0; li < nlev; ++li) {
      HostLevel& H = M.lv[li];
      H.nB = n_interior[li];
      H.nBb = n_boundary[li];
      H.brick_first = rows;
      rows += H.nB + H.nBb;
    }
    M.brick_nb.resize((size_t)rows * 27);
    for (int li = 0; li < nlev; ++li) {
      const HostLevel& H = M.lv[li];
      for (int64_t b = 0; b < H.nB + H.nBb; ++b)
        for (int t = 0; t < 27; ++t) {
          const int64_t pos = brick_nbpos[li][b][t];
          M.brick_nb[(size_t)(H.brick_first + b) * 27 + t] =
              pos == kMissingPos ? kBrickMissing : (int32_t)(pos - 64 * b);
        }
    }
    M.brick_tab.assign((size_t)(Q - 1) * 64, 0);
    for (int i = 1; i < Q; ++i)
      for (int l = 0; l < 64; ++l) {
        int64_t x[3] = {0, 0, 0};
        for (int bb = 0; bb < bshift; ++bb)
          for (int a = 0; a < d; ++a) x[a] |= (int64_t)((l >> (d * bb + a)) & 1) << bb;
        int t = 0, mul = 1;
        int64_t y[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a) {
          const int64_t q = a < d ? x[a] - B.dr.c[i][a] : 0;
          const int sa = q < 0 ? -1 : (q >= bside ? 1 : 0);
          y[a] = q - sa * bside;
          t += (sa + 1) * mul;
          mul *= 3;
        }
        M.brick_tab[(size_t)(i - 1) * 64 + l] = (uint16_t)((t << 6) | (int)zkey(y, d, bshift));
      }
    // the two-element BF16 kernel pulls both sources of positions 2m, 2m+1
    // through a link with c_x = 0 as one pair: same slot, positions l', l'+1
    for (int i = 1; i < Q; ++i) {
      if (B.dr.c[i][0] != 0) continue;
      for (int l = 0; l < 64; l += 2) {
        const uint16_t e0 = M.brick_tab[(size_t)(i - 1) * 64 + l], e1 = M.brick_tab[(size_t)(i - 1) * 64 + l + 1];
        if ((e0 & 1) || e1 != e0 + 1) return bad(LBM_ERR_INTERNAL, "brick link table breaks the x pairing");
      }
    }
  }
  // relaxation per level, Eq. (fneq_scale)
  M.lv[0].omega = p.omega_coarse;
  for (int li = 1; li < nlev; ++li) M.lv[li].omega = finer_omega(M.lv[li - 1].omega, B.mode);
  for (int li = 0; li < nlev; ++li)
    if (std::fabs(1.0 - M.lv[li].omega) < 1e-3) return bad(LBM_ERR_ARG, "omega too close to 1 on some level");

  // local indices into the grids; kinds
  M.kind.assign(M.Ntot, K_PAD);
  for (int li = 0; li < nlev; ++li) {
    HostLevel& H = M.lv[li];
    Grid& G = B.grid[li];
    std::vector<uint8_t>& kd = B.kind[li];
    kd.assign(H.N, K_PAD);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < H.nF; ++r) {
      G.g[G.at(&X[3 * fl[li][r].second])] = (int32_t)(H.oF + r);
      kd[H.oF + r] = K_FLUID;
    }
    for (int64_t k = 0; k < (int64_t)gff[li].size(); ++k) {
      const int64_t idx = k < H.nG1 ? H.oG1 + k : H.oG2 + (k - H.nG1);
      G.g[G.at(gff[li][k].x)] = (int32_t)idx;
      kd[idx] = K_GFF;
    }
    for (int64_t k = 0; k < H.nC; ++k) {
      int64_t o = G.at(gfc[li][k].x);
      if (o < 0) return bad(LBM_ERR_INTERNAL, "ghost outside its lookup grid");
      if (G.g[o] != G_NONE) return bad(LBM_ERR_MESH, "GhostFromCoarser collides with another element");
      G.g[o] = (int32_t)(H.oC + k);
      kd[H.oC + k] = K_GFC;
    }
    for (int64_t e = 0; e < H.N; ++e) M.kind[H.base + e] = kd[e];
    // host info of the ghosts
    H.ghost_xyz.resize(3 * (H.nC + H.nG1 + H.nG2));
    H.ghost_layer.resize(H.nC + H.nG1 + H.nG2);
    for (int64_t k = 0; k < H.nC; ++k) {
      for (int a = 0; a < 3; ++a) H.ghost_xyz[3 * k + a] = (int32_t)gfc[li][k].x[a];
      H.ghost_layer[k] = (int8_t)gfc[li][k].layer;
    }
    for (int64_t k = 0; k < (int64_t)gff[li].size(); ++k) {
      for (int a = 0; a < 3; ++a) H.ghost_xyz[3 * (H.nC + k) + a] = (int32_t)gff[li][k].x[a];
      H.ghost_layer[H.nC + k] = (int8_t)gff[li][k].layer;
    }
  }

  // GhostFromFiner children (contiguous siblings in z-curve order on level L+1)
  for (int li = 0; li + 1 < nlev; ++li) {
    HostLevel& H = M.lv[li];
    const HostLevel& Hf = M.lv[li + 1];
    H.gff_child0.resize(gff[li].size());
    for (size_t k = 0; k < gff[li].size(); ++k) {
      const Ghost& g = gff[li][k];
      int32_t first = -1;
      for (int b = 0; b < (1 << d); ++b) {
        int64_t c[3] = {2 * g.x[0] + (b & 1), 2 * g.x[1] + ((b >> 1) & 1), d == 3 ? 2 * g.x[2] + ((b >> 2) & 1) : 0};
        int32_t v = B.value(li + 1, c);
        if (v < 0 || B.kind[li + 1][v] != K_FLUID) return bad(LBM_ERR_MESH, "GhostFromFiner child is not a fluid element");
        if (b == 0) first = v;
        else if (v != first + b) return bad(LBM_ERR_INTERNAL, "GhostFromFiner children not contiguous");
      }
      H.gff_child0[k] = (int32_t)(Hf.base + first);
    }
  }

  // GhostFromCoarser sources on level L-1 (Sec. 2.2): parent H and, in the
  // ghost's octant, K(1,1,0), M(1,0,1), N(0,1,1); in 2D the square H, E, N, NE.
  for (int li = 1; li < nlev; ++li) {
    HostLevel& H = M.lv[li];
    HostLevel& Hc = M.lv[li - 1];
    static const int off3[4][3] = {{0, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
    static const int off2[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {1, 1, 0}};
    std::vector<int32_t> local(4 * H.nC);
    std::vector<int32_t> pos(Hc.N, -1);
    for (int64_t k = 0; k < H.nC; ++k) {
      const Ghost& g = gfc[li][k];
      int64_t P[3] = {g.x[0] >> 1, g.x[1] >> 1, g.x[2] >> 1};
      int sg[3];
      for (int a = 0; a < 3; ++a) sg[a] = ((g.oct >> a) & 1) ? 1 : -1;
      for (int s = 0; s < 4; ++s) {
        const int* o = d == 3 ? off3[s] : off2[s];
        int64_t q[3] = {P[0] + sg[0] * o[0], P[1] + sg[1] * o[1], d == 3 ? P[2] + sg[2] * o[2] : 0};
        int32_t v = B.wrap(li - 1, q) ? G_NONE : B.value(li - 1, q);
        if (v < 0 || B.kind[li - 1][v] == K_GFC || B.kind[li - 1][v] == K_PAD)
          return bad(LBM_ERR_MESH, "GhostFromCoarser source is neither fluid nor GhostFromFiner");
        local[4 * k + s] = v;
        pos[v] = 0;
      }
      H.gfc_oct.push_back(g.oct);
    }
    int32_t np = 0;
    for (int64_t e = 0; e < Hc.N; ++e)
      if (pos[e] == 0) {
        pos[e] = np++;
        Hc.src_elem.push_back((int32_t)(Hc.base + e));
      }
    H.gfc_src.resize(4 * H.nC);
    for (int64_t k = 0; k < H.nC; ++k)
      for (int s = 0; s < 4; ++s) H.gfc_src[s * H.nC + k] = pos[local[4 * k + s]];
    // the fill kernel takes the ghosts in sibling groups (octant = k mod 2^d)
    // whose sources depend only on the octant bits along their offsets
    const int G = 1 << d;
    if (H.nC % G) return bad(LBM_ERR_INTERNAL, "GhostFromCoarser ghosts not in complete sibling groups");
    for (int64_t k = 0; k < H.nC; ++k) {
      const int b = (int)(k % G);
      const int64_t k0 = k - b;
      // the sibling with the same bits along each source's offset and zeros elsewhere
      const int canon[4] = {0, d == 3 ? (b & 3) : (b & 1), d == 3 ? (b & 5) : (b & 2), d == 3 ? (b & 6) : (b & 3)};
      bool ok = H.gfc_oct[k] == b;
      for (int s = 0; s < 4 && ok; ++s) ok = H.gfc_src[s * H.nC + k] == H.gfc_src[s * H.nC + k0 + canon[s]];
      if (!ok) return bad(LBM_ERR_INTERNAL, "GhostFromCoarser sibling group inconsistent");
    }
    // bit 7 marks the outer layer (no fluid or subdivided cell on this level
    // within nlay - 1 cells)
    for (int64_t k = 0; k < H.nC; ++k)
      if (gfc[li][k].layer == nlay) H.gfc_oct[k] |= kGfcOuter;
  }
  // source bits per 32 slots (records written by the stream-collide) and the
  // GhostFromFiner sources (records written after the ghost fill)
  M.src_mask.assign((size_t)(M.Ntot / 32), 0u);
  M.src_first.assign((size_t)(M.Ntot / 32), 0);
  for (int li = 0; li < nlev; ++li) {
    HostLevel& H = M.lv[li];
    std::vector<int32_t> outer_e, outer_r;
    for (int64_t k = 0; k < (int64_t)H.src_elem.size(); ++k) {
      const int64_t e = H.src_elem[k];
      const size_t blk = (size_t)(e >> 5);
      if (!M.src_mask[blk]) M.src_first[blk] = (int32_t)k;
      M.src_mask[blk] |= 1u << (e & 31);
      if (M.kind[e] != K_GFF) continue;
      if (e - H.base < H.oG2) {
        H.gsrc_elem.push_back((int32_t)e);
        H.gsrc_rec.push_back((int32_t)k);
      } else {
        outer_e.push_back((int32_t)e);
        outer_r.push_back((int32_t)k);
      }
    }
    H.n_gsrc_inner = (int64_t)H.gsrc_elem.size();
    H.gsrc_elem.insert(H.gsrc_elem.end(), outer_e.begin(), outer_e.end());
    H.gsrc_rec.insert(H.gsrc_rec.end(), outer_r.begin(), outer_r.end());
  }

  // ---- pull neighbour lists (Sec. 2.1) with boundary rules (Sec. 2.3)
  M.nbr.assign((size_t)(Q - 1) * M.Ntot, 0);
  struct OutLink { int64_t e; int i, kind; int32_t a, b; };
  struct ObsLink { int64_t e; int i; int32_t a; };
  struct InLink { int64_t e; int i; double s; };
  std::vector<std::vector<OutLink>> outl(nlev);
  std::vector<std::vector<ObsLink>> obsl(nlev);
  std::vector<std::vector<InLink>> inl_(nlev);
  int inlet_axis = -1;
  for (int f = 0; f < 2 * d; ++f)
    if (B.bc[f] == LBM_BC_VELOCITY_IN) inlet_axis = f / 2;
  for (int li = 0; li < nlev; ++li) {
    const HostLevel& H = M.lv[li];
    const std::vector<uint8_t>& kd = B.kind[li];
    // element coordinates by local index
    std::vector<int64_t> pos(3 * H.N, 0);
    for (int64_t r = 0; r < H.nF; ++r)
      for (int a = 0; a < 3; ++a) pos[3 * (H.oF + r) + a] = X[3 * fl[li][r].second + a];
    for (int64_t k = 0; k < H.nC; ++k)
      for (int a = 0; a < 3; ++a) pos[3 * k + a] = gfc[li][k].x[a];
    for (int64_t k = 0; k < (int64_t)gff[li].size(); ++k) {
      const int64_t idx = k < H.nG1 ? H.oG1 + k : H.oG2 + (k - H.nG1);
      for (int a = 0; a < 3; ++a) pos[3 * idx + a] = gff[li][k].x[a];
    }
    std::vector<int8_t> layer(H.N, 0);
    for (int64_t k = 0; k < H.nC; ++k) layer[k] = (int8_t)gfc[li][k].layer;
    for (int64_t k = 0; k < H.nG1; ++k) layer[H.oG1 + k] = 1;
    std::vector<std::vector<OutLink>> po;
    std::vector<std::vector<ObsLink>> pb;
    std::vector<std::vector<InLink>> pi;
    int failed = 0;
    std::string ferr;
#pragma omp parallel
    {
#ifdef _OPENMP
      const int nt = omp_get_num_threads(), tid_ = omp_get_thread_num();
#else
      const int nt = 1, tid_ = 0;
#endif
#pragma omp single
      {
        po.resize(nt);
        pb.resize(nt);
        pi.resize(nt);
      }
      std::vector<OutLink> myo;
      std::vector<ObsLink> myb;
      std::vector<InLink> myi;
      std::string myerr;
#pragma omp for schedule(static)
      for (int64_t e = 0; e < H.N; ++e) {
        const uint8_t k = kd[e];
        const int64_t ge = H.base + e;
        // processed: fluid always; GFC (all layers) in TWO_LAYER and DIFFUSIVE
        // modes; inner GFF in LINEAR mode
        const bool proc = k == K_FLUID || (k == K_GFC && B.mode != LBM_TIME_LINEAR) ||
                          (k == K_GFF && layer[e] == 1 && B.mode == LBM_TIME_LINEAR);
        // ghosts whose pulled values reach fluid must find every neighbour: the
        // GFC layers before the outermost (whose processed values reach no
        // fluid before the next fill) and the GFF ghosts
        const bool strict_ghost = (k == K_GFC && layer[e] < nlay) || k == K_GFF;
        for (int i = 1; i < Q; ++i) {
          // default for links whose value never reaches a fluid element: read the
          // element's own opposite slot (each pdf slot keeps a single reader, so
          // the reverse of the streaming has no write conflicts)
          uint32_t code = proc ? NB_BOUNCE : (uint32_t)ge;
          if (proc) {
            int64_t q[3] = {pos[3 * e] - B.dr.c[i][0], pos[3 * e + 1] - B.dr.c[i][1], pos[3 * e + 2] - B.dr.c[i][2]};
            const int fc = B.wrap(li, q);
            if (fc) {
              if (k != K_FLUID) {
                if (strict_ghost) myerr = "ghost element next to the domain boundary";
              } else {
                bool wall = false, inl = false;
                int nout = 0, oface = -1;
                for (int f = 0; f < 2 * d; ++f) {
                  if (!(fc & (1 << f))) continue;
                  if (B.bc[f] == LBM_BC_WALL) wall = true;
                  if (B.bc[f] == LBM_BC_VELOCITY_IN) inl = true;
                  if (B.bc[f] == LBM_BC_PRESSURE_OUT) {
                    ++nout;
                    oface = f;
                  }
                }
                if (wall) {
                  code = NB_BOUNCE;
                } else if (inl) {
                  // inlet profile factor at the boundary point x - c_i / 2
                  double sf = 1.0;
                  if (p.inlet_profile == LBM_INLET_PARABOLIC)
                    for (int a = 0; a < d; ++a) {
                      if (a == inlet_axis) continue;
                      const double t = ((double)pos[3 * e + a] + 0.5 - 0.5 * B.dr.c[i][a]) / (double)B.ext(li, a);
                      sf *= 6.0 * t * (1.0 - t);
                    }
                  myi.push_back({ge, i, sf});
                  code = NB_BOUNCE | NB_FLAG30;  // index filled in after merging
                } else if (nout != 1) {
                  myerr = "outlet corner without wall";
                } else {
                  const int a = oface / 2, sg = (oface & 1) ? 1 : -1;
                  int nrm[3] = {0, 0, 0};
                  nrm[a] = sg;
                  const bool normal = B.dr.c[i][0] == -nrm[0] && B.dr.c[i][1] == -nrm[1] && B.dr.c[i][2] == -nrm[2];
                  OutLink ol{ge, i, normal ? OUT_NORMAL : OUT_EXTRAP, -1, -1};
                  if (!normal) {
                    // the outside element at x - c_i, extrapolated along -n
                    int64_t pa[3], pb2[3];
                    for (int c = 0; c < 3; ++c) {
                      const int64_t out_c = pos[3 * e + c] - B.dr.c[i][c];
                      pa[c] = out_c - nrm[c];
                      pb2[c] = out_c - 2 * nrm[c];
                    }
                    int32_t va = B.wrap(li, pa) ? G_NONE : B.value(li, pa);
                    int32_t vb = B.wrap(li, pb2) ? G_NONE : B.value(li, pb2);
                    if (va < 0 || vb < 0 || kd[va] != K_FLUID || kd[vb] != K_FLUID)
                      myerr = "outlet extrapolation source missing";
                    else {
                      ol.a = (int32_t)(H.base + va);
                      ol.b = (int32_t)(H.base + vb);
                    }
                  }
                  myo.push_back(ol);
                  code = NB_FLAG30;  // index filled in after merging
                }
              }
            } else {
              const int32_t v = B.value(li, q);
              if (v >= 0) {
                code = (uint32_t)(H.base + v);
                // the outer GhostFromCoarser layer is not refilled by the
                // LINEAR-mode step, so nothing processed may read it
                if (B.mode == LBM_TIME_LINEAR && kd[v] == K_GFC && layer[v] == 2)
                  myerr = "a processed element reads the outer GhostFromCoarser layer";
              } else if (k == K_FLUID) {
                if (v == G_SUB || B.covered_by_coarser(li, q))
                  myerr = "neighbour on another level has no ghost element";
                else {
                  // second node of the interpolated bounce-back: the element
                  // behind x, away from the wall (any element of this level)
                  int64_t pa[3] = {pos[3 * e] + B.dr.c[i][0], pos[3 * e + 1] + B.dr.c[i][1],
                                   pos[3 * e + 2] + B.dr.c[i][2]};
                  const int32_t va = B.wrap(li, pa) ? G_NONE : B.value(li, pa);
                  const int32_t a2 = va >= 0 ? (int32_t)(H.base + va) : -1;
                  myb.push_back({ge, i, a2});
                  if (p.bouzidi) {
                    myo.push_back({ge, i, OUT_BOUZIDI, a2, -1});
                    code = NB_FLAG30;  // index filled in after merging
                  } else {
                    code = NB_BOUNCE;
                  }
                }
              } else if (strict_ghost) {
                myerr = "ghost element next to a solid or missing neighbour";
              }
            }
          }
          M.nbr[(size_t)(i - 1) * M.Ntot + ge] = code;
        }
      }
#pragma omp critical
      {
        po[tid_].swap(myo);
        pb[tid_].swap(myb);
        pi[tid_].swap(myi);
        if (!myerr.empty()) {
          failed = 1;
          if (ferr.empty()) ferr = myerr;
        }
      }
    }
    if (failed) return bad(LBM_ERR_MESH, ferr);
    for (auto& v : po) outl[li].insert(outl[li].end(), v.begin(), v.end());
    for (auto& v : pb) obsl[li].insert(obsl[li].end(), v.begin(), v.end());
    for (auto& v : pi) inl_[li].insert(inl_[li].end(), v.begin(), v.end());
    std::sort(inl_[li].begin(), inl_[li].end(),
              [](const InLink& a, const InLink& b) { return a.e != b.e ? a.e < b.e : a.i < b.i; });
    std::sort(outl[li].begin(), outl[li].end(),
              [](const OutLink& a, const OutLink& b) { return a.e != b.e ? a.e < b.e : a.i < b.i; });
    std::sort(obsl[li].begin(), obsl[li].end(),
              [](const ObsLink& a, const ObsLink& b) { return a.e != b.e ? a.e < b.e : a.i < b.i; });
  }
  for (int li = 0; li < nlev; ++li) {
    HostLevel& H = M.lv[li];
    H.out_begin = (int64_t)M.out_elem.size();
    std::unordered_map<int64_t, int64_t> side_of;  // (element, direction) -> boundary-value index
    for (const OutLink& o : outl[li]) {
      const int64_t idx = (int64_t)M.out_elem.size();
      M.nbr[(size_t)(o.i - 1) * M.Ntot + o.e] = NB_FLAG30 | (uint32_t)idx;
      M.out_elem.push_back((int32_t)o.e);
      M.out_dir.push_back((int8_t)o.i);
      M.out_kind.push_back((int8_t)o.kind);
      M.out_a.push_back(o.a);
      M.out_b.push_back(o.b);
      M.out_q.push_back(0.5);
      if (o.kind == OUT_BOUZIDI) side_of[o.e * 32 + o.i] = idx;
    }
    H.out_end = (int64_t)M.out_elem.size();
    H.obs_begin = (int64_t)M.obs_elem.size();
    for (const ObsLink& o : obsl[li]) {
      M.obs_elem.push_back((int32_t)o.e);
      M.obs_dir.push_back((int8_t)o.i);
      M.obs_a.push_back(o.a);
      M.obs_q.push_back(0.5);
      auto it = side_of.find(o.e * 32 + o.i);
      M.obs_side.push_back(it == side_of.end() ? -1 : (int32_t)it->second);
    }
    H.obs_end = (int64_t)M.obs_elem.size();
    for (const InLink& o : inl_[li]) {
      const int64_t idx = (int64_t)M.inlet_s.size();
      M.nbr[(size_t)(o.i - 1) * M.Ntot + o.e] = NB_BOUNCE | NB_FLAG30 | (uint32_t)idx;
      M.inlet_s.push_back(o.s);
    }
  }
  if ((int64_t)M.inlet_s.size() >= (int64_t)NB_INDEX) return bad(LBM_ERR_MESH, "too many inlet links");
  if ((int64_t)M.out_elem.size() >= (int64_t)NB_INDEX) return bad(LBM_ERR_MESH, "too many outlet links");
  // every code the kernels decode stays inside its table, and every element
  // index of the boundary tables is -1 or an element
  {
    const uint64_t nout = M.out_elem.size(), nin = M.inlet_s.size();
    int badc = 0;
#pragma omp parallel for schedule(static) reduction(| : badc)
    for (int64_t k = 0; k < (int64_t)M.nbr.size(); ++k) {
      const uint32_t c = M.nbr[k];
      if (c < NB_FLAG30) badc |= (int64_t)c >= M.Ntot;
      else if ((c & NB_BOUNCE) && (c & NB_FLAG30)) badc |= (uint64_t)(c & NB_INDEX) >= nin;
      else if (!(c & NB_BOUNCE)) badc |= (uint64_t)(c & NB_INDEX) >= nout;
    }
    auto in_range = [&](const std::vector<int32_t>& v) {
      for (int32_t x : v)
        if (x < -1 || (int64_t)x >= M.Ntot) return false;
      return true;
    };
    if (badc || !in_range(M.out_elem) || !in_range(M.out_a) || !in_range(M.out_b) || !in_range(M.obs_elem) ||
        !in_range(M.obs_a))
      return bad(LBM_ERR_INTERNAL, "boundary table index out of range");
  }
  // brick links must reproduce the neighbour list exactly (boundary bricks:
  // every link not routed to the neighbour list; interior bricks: all links)
  for (int li = 0; li < nlev; ++li) {
    const HostLevel& H = M.lv[li];
    int mismatch = 0;
#pragma omp parallel for schedule(static) reduction(| : mismatch)
    for (int64_t b = 0; b < H.nB + H.nBb; ++b) {
      const int32_t* nb = &M.brick_nb[(size_t)(H.brick_first + b) * 27];
      for (int i = 1; i < Q; ++i)
        for (int l = 0; l < 64; ++l) {
          const uint16_t v = M.brick_tab[(size_t)(i - 1) * 64 + l];
          const int64_t first = H.base + H.oF + 64 * b;
          if (nb[v >> 6] == kBrickMissing) {
            if (b < H.nB) mismatch = 1;
            continue;
          }
          if (M.nbr[(size_t)(i - 1) * M.Ntot + first + l] != (uint32_t)(first + nb[v >> 6] + (v & 63))) mismatch = 1;
        }
    }
    if (mismatch) return bad(LBM_ERR_INTERNAL, "brick table disagrees with the neighbour list");
  }

  // ---- caller order <-> element slots
  M.uslot.resize(n);
  M.ulev.resize(n);
  M.slot_user.assign(M.Ntot, -1);
  for (int li = 0; li < nlev; ++li) {
    const HostLevel& H = M.lv[li];
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < H.nF; ++r) {
      const int64_t k = fl[li][r].second;
      M.uslot[k] = (int32_t)(H.base + H.oF + r);
      M.ulev[k] = (uint8_t)li;
      M.slot_user[H.base + H.oF + r] = (int32_t)k;
    }
  }
  return LBM_OK;
}

// Sec. 3.1: z-curve order over mixed levels (a coarse element precedes its
// finer neighbours in the order of its first corner at the finest level),
// weights w = 2^{L - Lmin}, cumulative W, equal-share split into nparts.
lbm_status sfc_partition(const int64_t* tid, int64_t n, int d, int nparts, int64_t* order,
                         int64_t* weights, int64_t* cumulative, int32_t* part, std::string* msg) {
  if (!tid || n <= 0 || (d != 2 && d != 3) || nparts < 1) {
    *msg = "bad argument";
    return LBM_ERR_ARG;
  }
  std::vector<int> L(n);
  std::vector<int64_t> X(3 * n);
  for (int64_t k = 0; k < n; ++k)
    if (!decode_tid(tid[k], d, &L[k], &X[3 * k])) {
      *msg = "invalid treeID";
      return LBM_ERR_MESH;
    }
  const int Lmin = *std::min_element(L.begin(), L.end());
  const int Lmax = *std::max_element(L.begin(), L.end());
  std::vector<std::pair<uint64_t, int64_t>> key(n);
  for (int64_t k = 0; k < n; ++k) {
    int64_t c[3];
    for (int a = 0; a < 3; ++a) c[a] = X[3 * k + a] << (Lmax - L[k]);
    key[k] = {zkey(c, d, Lmax), k};
  }
  std::sort(key.begin(), key.end());
  int64_t W = 0;
  std::vector<int64_t> cum(n);
  for (int64_t r = 0; r < n; ++r) {
    const int64_t w = (int64_t)1 << (L[key[r].second] - Lmin);
    W += w;
    cum[r] = W;
    if (order) order[r] = key[r].second;
    if (weights) weights[r] = w;
    if (cumulative) cumulative[r] = W;
  }
  if (part)
    for (int64_t r = 0; r < n; ++r) {
      // element r goes to the first part whose share W*(p+1)/nparts it does not exceed
      int32_t pp = (int32_t)(((__int128)(cum[r] - 1) * nparts) / W);
      part[r] = std::min(pp, nparts - 1);
    }
  return LBM_OK;
}

}  // namespace lbm
