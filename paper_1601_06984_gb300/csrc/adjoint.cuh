// Discrete adjoint of the multilevel step (reverse mode, hand-written).
//
// Every forward kernel of the path has a reverse here: pull stream + BGK
// collide (Sec. 2.1), the outlet values (Sec. 2.3), the GhostFromCoarser
// source moments and compact interpolation and the GhostFromFiner restriction
// (Sec. 2.2).  A reverse kernel reads the forward state the op saw (a snapshot),
// consumes the adjoint of the op's outputs (and zeroes it: those slots were
// overwritten by the op), and adds the transposed Jacobian times that adjoint
// to the adjoint of the op's inputs.  Scatter targets are unique within one
// launch (each pdf slot is pulled by exactly one element; each ghost has its
// own children; each source element appears once), so plain read-modify-write
// is race-free; the ghost-to-source sums of GhostFromCoarser go through a
// transposed (CSR) list so that they are deterministic too.  Derivatives with
// respect to the relaxation rates and the inlet velocity are summed per block
// into the block's own running row (launches are stream-ordered) and the rows
// are summed once at the end, in block order (deterministic); body-force
// derivatives are accumulated per element in FP64.
#pragma once

#include "kernels.cuh"

namespace lbm {
namespace dev {

// Minimum resident blocks per SM of the reverse kernels with 4-byte compute
// type (FP64 keeps the lower counts, its registers being twice as many).
// Measured on the two-level TGV adjoint (FP32 deviation, 400 steps): three
// blocks of brick reverse (80 registers), two of GhostFromFiner reverse and
// four of moments reverse (128 registers, small spills) 0.214 s against
// 0.219 s with the compiler's choice; the list reverse spills 600 B at three.
#ifndef LBM_ADJ_SC_MINB
#define LBM_ADJ_SC_MINB 2
#endif
#ifndef LBM_ADJ_BRICK_MINB
#define LBM_ADJ_BRICK_MINB 3
#endif
#ifndef LBM_ADJ_MOM_MINB
#define LBM_ADJ_MOM_MINB 4
#endif
#ifndef LBM_ADJ_GFF_MINB
#define LBM_ADJ_GFF_MINB 2
#endif
#define LBM_ADJ_MINB(S, M, M64) (sizeof(typename Sto<S>::R) == 8 ? (M64) : (M))

// ----------------------------------------------------------------- reverse helpers
// Reverse of g^eq_i(rp, rho = rho_off + rp, u) for all i, weighted by lam[i]:
// adds to lam_rp and lam_u.
template <int Q, class R>
__device__ __forceinline__ void geq_rev(const R* lam, R rho, const R* u, R usq, R& lam_rp, R* lam_u) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    R cu = R(0);
#pragma unroll
    for (int a = 0; a < D; ++a) cu += R(LT::c(i, a)) * u[a];
    const R wl = R(LT::w(i)) * lam[i];
    lam_rp += wl * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq);
    const R t = wl * rho;
#pragma unroll
    for (int a = 0; a < D; ++a) lam_u[a] += t * (R(3) * R(LT::c(i, a)) + R(9) * cu * R(LT::c(i, a)) - R(3) * u[a]);
  }
}

// Reverse of the Guo term (1 - omega/2) w_i [3 (c_i.F - u.F) + 9 (c_i.u)(c_i.F)].
template <int Q, class R>
__device__ __forceinline__ void guo_rev(const R* lam, R om, const R* u, const R* F, R& lam_om, R* lam_u, R* lam_F) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  const R pre = R(1) - R(0.5) * om;
  R uF = R(0);
#pragma unroll
  for (int a = 0; a < D; ++a) uF += u[a] * F[a];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    R cu = R(0), cF = R(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      cu += R(LT::c(i, a)) * u[a];
      cF += R(LT::c(i, a)) * F[a];
    }
    const R wl = R(LT::w(i)) * lam[i];
    lam_om += -R(0.5) * wl * (R(3) * (cF - uF) + R(9) * cu * cF);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const R ca = R(LT::c(i, a));
      lam_u[a] += pre * wl * (-R(3) * F[a] + R(9) * ca * cF);
      lam_F[a] += pre * wl * (R(3) * (ca - u[a]) + R(9) * cu * ca);
    }
  }
}

// Reverse of post_moments (stored post-collision pdfs -> rp, u, f^neq, S).
// Inputs: the pdfs g, the adjoints of the outputs (lam_fneq is overwritten).
// Outputs: lam_g (assigned), lam_F and lam_om (accumulated).
template <int Q, class R>
__device__ __forceinline__ void post_moments_rev(const R* g, R om, R rho_off, const R* F, R lam_rp_in,
                                                 const R* lam_u_in, R* lam_fneq, const R* lam_S, R* lam_g,
                                                 R* lam_F, R& lam_om) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  R rp, j[3];
  raw_moments<Q, R>(g, rp, j);
  const R rho = rho_off + rp;
  const R inv = R(1) / rho;
  R u[3] = {R(0), R(0), R(0)};
  R usq = R(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    u[a] = (j[a] - R(0.5) * F[a]) * inv;
    usq += u[a] * u[a];
  }
  const R r1w = R(1) / (R(1) - om);
  R fneq[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) fneq[i] = (g[i] - geq<Q, R>(i, rp, rho, u, usq) - guo<Q, R>(i, om, u, F)) * r1w;
  const R pre = -R(1.5) * om * inv;
  R lam_pre = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    R add = R(0);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = a; b < D; ++b) {
        const int cc = LT::c(i, a) * LT::c(i, b);
        if (cc != 0) {
          const R ls = lam_S[sidx<D>(a, b)];
          add += R(cc) * ls;
          lam_pre += R(cc) * ls * fneq[i];
        }
      }
    lam_fneq[i] += pre * add;
  }
  R lam_rho = lam_pre * R(1.5) * om * inv * inv;
  lam_om += lam_pre * (-R(1.5) * inv);
  R lam_rp = lam_rp_in;
  R lam_u[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int a = 0; a < D; ++a) lam_u[a] = lam_u_in[a];
  R lam_q[Q];
  R lam_r1w = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    lam_g[i] = lam_fneq[i] * r1w;
    lam_q[i] = -lam_fneq[i] * r1w;
    lam_r1w += lam_fneq[i] * fneq[i];  // fneq = (...) r1w, so d/dr1w = fneq / r1w
  }
  lam_om += lam_r1w * r1w;  // d r1w / d omega = r1w^2; times fneq/r1w gives fneq * r1w
  guo_rev<Q, R>(lam_q, om, u, F, lam_om, lam_u, lam_F);
  geq_rev<Q, R>(lam_q, rho, u, usq, lam_rp, lam_u);
  R lam_j[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    lam_j[a] = lam_u[a] * inv;
    lam_F[a] += -R(0.5) * lam_u[a] * inv;
    lam_rho += -lam_u[a] * u[a] * inv;
  }
  lam_rp += lam_rho;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    R v = lam_g[i] + lam_rp;
#pragma unroll
    for (int a = 0; a < D; ++a) v += R(LT::c(i, a)) * lam_j[a];
    lam_g[i] = v;
  }
}

// Reverse of one element's BGK collision with Guo forcing (u = (j + F/2) / rho),
// from the pdfs g it pulled and the adjoints lo of its outputs.  The collision
// Jacobian is the identity times (1 - omega) plus a rank-(1+d) part: with
//   A_i = d g^eq_i / d rp,  B_ia = d g^eq_i / d u_a,  G_ia = d guo_i / d u_a,
//   S0 = sum_i lo_i A_i,   S_a = sum_i lo_i (omega B_ia + G_ia),
// the adjoint of pulled pdf i is
//   lam_g_i = (1 - omega) lo_i + base + sum_a c_ia sa_a,
//   base = omega S0 - sum_a S_a u_a / rho,  sa_a = S_a / rho.
// Every sum over i is linear in P_i = w_i lo_i with weights of degree <= 2 in
// c_i, so it is formed from M0 = sum P_i, M1_a = sum P_i c_ia and
// M2_ab = sum P_i c_ia c_ib.  lF and lom receive the element's derivatives with
// respect to its force and omega.
template <int Q, class R>
__device__ __forceinline__ void bgk_rev(const R* g, const R* lo, const R* F, R om, R rho_off, R& base, R* sa,
                                        R* lF, R& lom) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  R rp, j[3];
  raw_moments<Q, R>(g, rp, j);
  const R rho = rho_off + rp, inv = R(1) / rho;
  R u[3] = {R(0), R(0), R(0)}, usq = R(0), uF = R(0);
#pragma unroll
  for (int b = 0; b < D; ++b) {
    u[b] = (j[b] + R(0.5) * F[b]) * inv;
    usq += u[b] * u[b];
    uF += u[b] * F[b];
  }
  const R fpre = R(1) - R(0.5) * om;
  R M0 = R(0), M1[3] = {R(0), R(0), R(0)}, M2[3][3] = {}, lg_dot = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const R P = R(LT::w(i)) * lo[i];
    lg_dot += lo[i] * g[i];
    M0 += P;
#pragma unroll
    for (int b = 0; b < D; ++b) {
      if (LT::c(i, b) > 0) M1[b] += P;
      if (LT::c(i, b) < 0) M1[b] -= P;
#pragma unroll
      for (int c = b; c < D; ++c) {
        const int cc = LT::c(i, b) * LT::c(i, c);
        if (cc > 0) M2[b][c] += P;
        if (cc < 0) M2[b][c] -= P;
      }
    }
  }
  R M2u[3] = {R(0), R(0), R(0)}, M2F[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int b = 0; b < D; ++b)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const R m = b <= c ? M2[b][c] : M2[c][b];
      M2u[b] += m * u[c];
      M2F[b] += m * F[c];
    }
  R uM1 = R(0), FM1 = R(0), uM2u = R(0), uM2F = R(0);
#pragma unroll
  for (int b = 0; b < D; ++b) {
    uM1 += u[b] * M1[b];
    FM1 += F[b] * M1[b];
    uM2u += u[b] * M2u[b];
    uM2F += u[b] * M2F[b];
  }
  // sum lo_i A_i, sum lo_i g^eq_i, sum lo_i Guo_i
  const R quad = R(3) * uM1 + R(4.5) * uM2u - R(1.5) * usq * M0;
  const R S0 = M0 + quad;
  const R sum_geq = rp * M0 + rho * quad;
  const R sum_G = R(3) * (FM1 - uF * M0) + R(9) * uM2F;
  lom = sum_geq - lg_dot - R(0.5) * sum_G;
  base = om * S0;
#pragma unroll
  for (int b = 0; b < D; ++b) {
    const R lin = R(3) * M1[b] + R(9) * M2u[b] - R(3) * u[b] * M0;  // sum lo_i B_ib / rho
    const R Sa = om * rho * lin + fpre * (R(9) * M2F[b] - R(3) * F[b] * M0);
    lF[b] = fpre * lin + R(0.5) * Sa * inv;
    base -= Sa * u[b] * inv;
    sa[b] = Sa * inv;
  }
}

// Adds the block's sums to its running row: v[0] to omega of level c.la, v[1]
// to omega of level c.lb, v[2..4] to u_in.
template <class R, int NV>
__device__ __forceinline__ void store_partials(R (&v)[NV], const AdjCommon& c) {
  __shared__ double tot[NV];
  double d[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) d[k] = (double)v[k];
  block_sum_store<NV>(d, tot);  // written by thread 0, which also reads them
  if (threadIdx.x == 0) {
    double* row = c.partial + (size_t)blockIdx.x * kAccCols;
    row[c.la] += tot[0];
    if (NV > 1 && c.lb >= 0) row[c.lb] += tot[NV > 1 ? 1 : 0];
#pragma unroll
    for (int b = 0; b < 3; ++b)
      if (NV > 2 + b) row[16 + b] += tot[NV > 2 + b ? 2 + b : 0];
  }
}

// Read-modify-writes below issue every load before the first store: the
// compiler cannot tell that rows q N + e of one array are distinct, and would
// otherwise wait for each load in turn.
template <class R>
__device__ __forceinline__ void add_force(double* lam_force, int64_t Ntot, int64_t e, const R* lF, int D) {
  if (!lam_force) return;
  double cur[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < D; ++b) cur[b] = lam_force[(size_t)b * Ntot + e];
  for (int b = 0; b < D; ++b) lam_force[(size_t)b * Ntot + e] = cur[b] + (double)lF[b];
}

// lam[q N + e] += v[q] for q < Q
template <int Q, class R>
__device__ __forceinline__ void add_rows(R* lam, size_t N, int64_t e, const R* v) {
  R cur[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) cur[q] = lam[(size_t)q * N + e];
#pragma unroll
  for (int q = 0; q < Q; ++q) lam[(size_t)q * N + e] = cur[q] + v[q];
}

template <class S, class R>
__device__ __forceinline__ void load_force(const void* force, int64_t Ntot, int64_t e, R* F, int D) {
  F[0] = F[1] = F[2] = R(0);
  if (force)
    for (int b = 0; b < D; ++b) F[b] = static_cast<const R*>(force)[(size_t)b * Ntot + e];
}

// ----------------------------------------------------------------- objective seeds
// Kinetic energy J = sum vol rho |u|^2 / 2 with rho u = j - F/2: dJ/dg_i =
// vol (c_i.u - |u|^2/2), dJ/dF = -vol u / 2.  Obstacle force component k:
// J = sum_links 2 fscale c_opp,k f*_opp  ->  dJ/dg_opp = 2 fscale c_opp,k.
template <int Q, class S>
__global__ void __launch_bounds__(256) k_adj_seed(const AdjSeedArgs a) {
  using R = typename Sto<S>::R;
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  const S* __restrict__ x = static_cast<const S*>(a.c.fsrc);
  R* lam = static_cast<R*>(a.c.lam_b);
  const size_t N = (size_t)a.c.Ntot;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a.objective == 0) {
    for (int64_t e = a.begin + t0; e < a.end; e += stride) {
      R g[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) g[q] = Sto<S>::ld(x + (size_t)q * N + e);
      R F[3];
      load_force<S, R>(a.c.force, a.c.Ntot, e, F, D);
      R rp, j[3];
      raw_moments<Q, R>(g, rp, j);
      const R rho = R(a.c.rho_off) + rp;
      R u[3] = {R(0), R(0), R(0)}, usq = R(0);
#pragma unroll
      for (int b = 0; b < D; ++b) {
        u[b] = (j[b] - R(0.5) * F[b]) / rho;
        usq += u[b] * u[b];
      }
      const R vol = R(a.vol);
      R v[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        R cu = R(0);
#pragma unroll
        for (int b = 0; b < D; ++b) cu += R(LT::c(q, b)) * u[b];
        v[q] = vol * (cu - R(0.5) * usq);
      }
      add_rows<Q, R>(lam, N, e, v);
      R lF[3];
#pragma unroll
      for (int b = 0; b < D; ++b) lF[b] = -R(0.5) * vol * u[b];
      add_force<R>(a.c.lam_force, a.c.Ntot, e, lF, D);
    }
  } else {
    // F_k = fscale c_ib,k (f*_ib(x) + f_i(x)), f_i the (interpolated) bounce-
    // back value: pass 0 seeds f*_ib(x), pass 1 f*_ib(x + c_i), pass 2 f*_i(x)
    const int k = a.objective - 1;
    for (int64_t l = t0; l < a.obs_n; l += stride) {
      const int i = a.obs_dir[l];
      const int ib = opp(i);
      const int64_t e = a.obs_elem[l];
      int cb = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q)
        if (q == ib) cb = LT::c(q, k < D ? k : 0);
      if (k >= D) continue;
      const double q = a.obs_q ? a.obs_q[l] : 0.5;
      const int32_t a2 = a.obs_a ? a.obs_a[l] : -1;
      double w_own, w_a = 0.0, w_i = 0.0;
      if (q < 0.5) {
        w_own = a2 < 0 ? 2.0 : 1.0 + 2.0 * q;
        if (a2 >= 0) w_a = 1.0 - 2.0 * q;
      } else {
        w_own = 1.0 + 1.0 / (2.0 * q);
        w_i = (2.0 * q - 1.0) / (2.0 * q);
      }
      const double base = a.fscale * cb;
      if (a.which == 0) lam[(size_t)ib * N + e] += R(base * w_own);
      if (a.which == 1 && w_a != 0.0) lam[(size_t)ib * N + a2] += R(base * w_a);
      if (a.which == 2 && w_i != 0.0) lam[(size_t)i * N + e] += R(base * w_i);
    }
  }
}

// ----------------------------------------------------------------- stream + collide
// Reverse of one element's pull + BGK collide through the neighbour list
// (every element the interior-brick kernel does not take): the pulled pdfs
// are gathered as the forward did, bgk_rev gives the adjoint of each, and it
// is added to the slot the forward pulled from (a conflict-free scatter: each
// slot has one reader), or to the adjoint of the outlet value it came from.
template <int Q, class S>
__global__ void __launch_bounds__(256, LBM_ADJ_MINB(S, LBM_ADJ_SC_MINB, 2)) k_adj_sc(const AdjSCArgs a) {
  using R = typename Sto<S>::R;
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  const S* __restrict__ x = static_cast<const S*>(a.c.fsrc);
  R* __restrict__ lam_out = static_cast<R*>(a.c.lam_a);
  R* __restrict__ lam_in = static_cast<R*>(a.c.lam_b);
  const size_t N = (size_t)a.c.Ntot;
  const R om = R(a.omega), rho_off = R(a.c.rho_off);
  R part[5] = {R(0), R(0), R(0), R(0), R(0)};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t lin = a.begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; lin < a.end; lin += stride) {
    const int64_t e = lin + (lin >= a.hole_at ? a.hole_len : 0);
    uint32_t nb[Q];
    nb[0] = (uint32_t)e;
#pragma unroll
    for (int i = 1; i < Q; ++i) nb[i] = __ldg(a.nbr + (size_t)(i - 1) * N + e);
    R g[Q];
    g[0] = Sto<S>::ld(x + e);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t n = nb[i];
      const size_t idx = n < NB_FLAG30 ? (size_t)i * N + n : (size_t)opp(i) * N + (size_t)e;
      g[i] = Sto<S>::ld(x + idx);
    }
    R lo[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) lo[i] = lam_out[(size_t)i * N + e];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t n = nb[i];
      if (n >= NB_FLAG30) {
        if (n & NB_BOUNCE) {
          if (n & NB_FLAG30) g[i] += R(a.inlet[i]) * (a.inlet_s ? R(a.inlet_s[n & NB_INDEX]) : R(1));
        } else {
          g[i] = static_cast<const R*>(a.side_fwd)[n & NB_INDEX];
        }
      }
    }
    R F[3];
    load_force<S, R>(a.c.force, a.c.Ntot, e, F, D);
    R base, sa[3] = {R(0), R(0), R(0)}, lF[3] = {R(0), R(0), R(0)}, lom;
    bgk_rev<Q, R>(g, lo, F, om, rho_off, base, sa, lF, lom);
    part[0] += lom;
    add_force<R>(a.c.lam_force, a.c.Ntot, e, lF, D);
    // the adjoints of the pulled pdfs replace lo (which nothing reads after)
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      R lg = (R(1) - om) * lo[i] + base;
#pragma unroll
      for (int b = 0; b < D; ++b) lg += sa[b] * R(LT::c(i, b));
      lo[i] = lg;
    }
    // reverse streaming
    auto target = [&](int i) -> size_t {
      const uint32_t n = nb[i];
      return i == 0 ? (size_t)e : (n < NB_FLAG30 ? (size_t)i * N + n : (size_t)opp(i) * N + (size_t)e);
    };
    R cur[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const bool side = i > 0 && nb[i] >= NB_FLAG30 && !(nb[i] & NB_BOUNCE);
      cur[i] = side ? R(0) : lam_in[target(i)];
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const R lg = lo[i];
      const uint32_t n = nb[i];
      lam_out[(size_t)i * N + e] = R(0);
      if (i > 0 && n >= NB_FLAG30 && !(n & NB_BOUNCE)) {
        static_cast<R*>(a.lam_side)[n & NB_INDEX] = lg;
        continue;
      }
      lam_in[target(i)] = cur[i] + lg;
      if (i > 0 && (n & NB_BOUNCE) && (n & NB_FLAG30)) {
        // d f_i / d u_in = 6 w_i rho0 s c_i, s the link's inlet profile factor
        const R sf = a.inlet_s ? R(a.inlet_s[n & NB_INDEX]) : R(1);
#pragma unroll
        for (int b = 0; b < D; ++b) part[2 + b] += lg * sf * R(6.0 * LT::w(i) * a.c.rho0 * LT::c(i, b));
      }
    }
  }
  store_partials<R, 5>(part, a.c);
}

// Reverse of the interior-brick stream + collide.  The forward kernel's pull:
// each group of 64 threads takes one brick (thread l its element at z-curve
// position l), and the pull source of link i is the brick's neighbour row
// entry for the thread's link-table slot plus the position in that brick.  The
// reverse gathers the same sources from the snapshot and scatters the pulled
// pdfs' adjoints back into those slots; interior bricks have no boundary
// links.  Grid: ceil(nB / 4) blocks of 256, block b adding its sums to running
// row b.
static_assert(LBM_BR_BLOCK / 64 == LBM_BRICKS_PER_BLOCK, "host sizes the running rows by this many bricks per block");
template <int Q, class S>
__global__ void __launch_bounds__(LBM_BR_BLOCK, LBM_ADJ_MINB(S, LBM_ADJ_BRICK_MINB, 2)) k_adj_sc_brick(const AdjSCArgs a) {
  using R = typename Sto<S>::R;
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  constexpr int BPB = LBM_BR_BLOCK / 64;
  constexpr int NW = Q / 2;  // (Q-1)/2 words of two 16-bit entries
  const int l = threadIdx.x & 63, lane = threadIdx.x & 31;
  // the brick index is uniform over each warp, so the shuffles run with whole warps
  const int64_t bk = (int64_t)blockIdx.x * BPB + (threadIdx.x >> 6);
  R part[1] = {R(0)};
  if (bk < a.nB) {
    uint32_t tw[NW];
#pragma unroll
    for (int k = 0; k < NW; ++k)
      tw[k] = (uint32_t)__ldg(a.brick_tab + (2 * k) * 64 + l) |
              ((uint32_t)__ldg(a.brick_tab + (2 * k + 1) * 64 + l) << 16);
    const int32_t row = lane < 27 ? __ldg(a.brick_nb + bk * 27 + lane) : 0;
    const size_t N = (size_t)a.c.Ntot;
    const int64_t first = a.begin + bk * 64, e = first + l;
    const S* __restrict__ x = static_cast<const S*>(a.c.fsrc) + first;
    R* __restrict__ lam_out = static_cast<R*>(a.c.lam_a);
    R* __restrict__ lam_in = static_cast<R*>(a.c.lam_b) + first;
    // pull source of link i: row i of the state, at this 32-bit offset from
    // the brick's first element (kept, not the 64-bit addresses)
    int32_t off[Q];
    off[0] = l;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t v = (tw[(i - 1) >> 1] >> (((i - 1) & 1) * 16)) & 0xffffu;
      off[i] = __shfl_sync(0xffffffffu, row, (int)(v >> 6)) + (int32_t)(v & 63);
    }
    R g[Q], lo[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = Sto<S>::ld(x + (int64_t)(i * N) + off[i]);
#pragma unroll
    for (int i = 0; i < Q; ++i) lo[i] = lam_out[(size_t)i * N + e];
    R F[3];
    load_force<S, R>(a.c.force, a.c.Ntot, e, F, D);
    const R om = R(a.omega);
    R base, sa[3] = {R(0), R(0), R(0)}, lF[3] = {R(0), R(0), R(0)}, lom;
    bgk_rev<Q, R>(g, lo, F, om, R(a.c.rho_off), base, sa, lF, lom);
    part[0] += lom;
    add_force<R>(a.c.lam_force, a.c.Ntot, e, lF, D);
    // the adjoints of the pulled pdfs replace lo (which nothing reads after)
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      R lg = (R(1) - om) * lo[i] + base;
#pragma unroll
      for (int b = 0; b < D; ++b) lg += sa[b] * R(LT::c(i, b));
      lo[i] = lg;
    }
    R cur[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) cur[i] = lam_in[(int64_t)(i * N) + off[i]];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      lam_out[(size_t)i * N + e] = R(0);
      lam_in[(int64_t)(i * N) + off[i]] = cur[i] + lo[i];
    }
  }
  store_partials<R, 1>(part, a.c);
}

// ----------------------------------------------------------------- outlet values
template <int Q, class S>
__global__ void __launch_bounds__(256) k_adj_outlet(const AdjOutletArgs a) {
  using R = typename Sto<S>::R;
  using LT = Lat<Q>;
  constexpr int D = LT::D, NS = LT::NS;
  const S* __restrict__ x = static_cast<const S*>(a.c.fsrc);
  R* lam_in = static_cast<R*>(a.c.lam_b);
  const R* lam_side = static_cast<const R*>(a.lam_side);
  const size_t N = (size_t)a.c.Ntot;
  R part[1] = {R(0)};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = a.begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.end; k += stride) {
    const int i = a.dir[k];
    const R ls = lam_side[k];
    if (a.kind[k] == OUT_EXTRAP) {
      if (a.which == 1) lam_in[(size_t)i * N + a.a[k]] += a.zero_gradient ? ls : R(2) * ls;
      if (a.which == 2 && !a.zero_gradient) lam_in[(size_t)i * N + a.b[k]] -= ls;
      continue;
    }
    if (a.kind[k] == OUT_BOUZIDI) {
      // interpolated bounce-back value, linear in f*_i(x) (pass 3), f*_ib(x)
      // (pass 4) and f*_ib(x + c_i) (pass 5); one slot per link and pass
      const int ib = opp(i);
      const int64_t e = a.elem[k];
      const double q = a.q ? a.q[k] : 0.5;
      const int32_t a2 = a.a[k];
      if (q < 0.5) {
        if (a.which == 4) lam_in[(size_t)ib * N + e] += a2 < 0 ? ls : R(2.0 * q) * ls;
        if (a.which == 5 && a2 >= 0) lam_in[(size_t)ib * N + a2] += R(1.0 - 2.0 * q) * ls;
      } else {
        if (a.which == 4) lam_in[(size_t)ib * N + e] += R(1.0 / (2.0 * q)) * ls;
        if (a.which == 3) lam_in[(size_t)i * N + e] += R((2.0 * q - 1.0) / (2.0 * q)) * ls;
      }
      continue;
    }
    if (a.which != 0) continue;
    // side = g^eq_i(rho0, u) + f^neq_ib, with u and the pre-collision f^neq
    // taken from the stored pdfs g (post_moments)
    const int64_t e = a.elem[k];
    R g[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) g[q] = Sto<S>::ld(x + (size_t)q * N + e);
    R F[3];
    load_force<S, R>(a.c.force, a.c.Ntot, e, F, D);
    R rp, j[3];
    raw_moments<Q, R>(g, rp, j);
    const R rho = R(a.c.rho_off) + rp, inv = R(1) / rho;
    R u[3] = {R(0), R(0), R(0)}, usq = R(0);
#pragma unroll
    for (int b = 0; b < D; ++b) {
      u[b] = (j[b] - R(0.5) * F[b]) * inv;
      usq += u[b] * u[b];
    }
    const int ib = opp(i);
    // term g^eq_i(rho0, u): depends on u only
    R lam_rp_dummy = R(0), lam_u[3] = {R(0), R(0), R(0)};
    R l1[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) l1[q] = q == i ? ls : R(0);
    geq_rev<Q, R>(l1, R(a.c.rho0), u, usq, lam_rp_dummy, lam_u);
    // term f^neq_ib, and u's dependence on g
    R lfn[Q], lS[NS], lg[Q], lF[3] = {R(0), R(0), R(0)}, lom = R(0);
#pragma unroll
    for (int q = 0; q < Q; ++q) lfn[q] = q == ib ? ls : R(0);
#pragma unroll
    for (int s2 = 0; s2 < NS; ++s2) lS[s2] = R(0);
    post_moments_rev<Q, R>(g, R(a.omega), R(a.c.rho_off), F, R(0), lam_u, lfn, lS, lg, lF, lom);
    add_rows<Q, R>(lam_in, N, e, lg);
    add_force<R>(a.c.lam_force, a.c.Ntot, e, lF, D);
    part[0] += lom;
  }
  if (a.which == 0) store_partials<R, 1>(part, a.c);
}

// ----------------------------------------------------------------- source moments
template <int Q, class S>
__global__ void __launch_bounds__(128, LBM_ADJ_MINB(S, LBM_ADJ_MOM_MINB, 1)) k_adj_moments(const AdjMomArgs a) {
  using R = typename Sto<S>::R;
  using LT = Lat<Q>;
  using RL = RecLayout<Q>;
  constexpr int D = LT::D, NS = LT::NS;
  const S* __restrict__ x = static_cast<const S*>(a.c.fsrc);
  R* lam_in = static_cast<R*>(a.c.lam_b);
  const size_t N = (size_t)a.c.Ntot;
  R part[1] = {R(0)};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.nsrc; k += stride) {
    R* __restrict__ lr = static_cast<R*>(a.lam_rec) + (size_t)k * RL::STRIDE;
    R rec[RL::STRIDE];
#pragma unroll
    for (int f = 0; f < RL::STRIDE; f += 4) ld4(lr + f, rec + f);
    if (a.lam_rec_prev) {
      // the record at t+1/2 is the mean of those at t and t+1
      R* __restrict__ lp = static_cast<R*>(a.lam_rec_prev) + (size_t)k * RL::STRIDE;
      R pv[RL::STRIDE];
#pragma unroll
      for (int f = 0; f < RL::STRIDE; f += 4) ld4(lp + f, pv + f);
#pragma unroll
      for (int f = 0; f < RL::STRIDE; ++f) {
        rec[f] *= R(0.5);
        pv[f] += rec[f];
      }
#pragma unroll
      for (int f = 0; f < RL::STRIDE; f += 4) st4(lp + f, pv + f);
    }
    {
      R z[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
      for (int f = 0; f < RL::STRIDE; f += 4) st4(lr + f, z);
    }
    const int64_t e = a.elem[k];
    R g[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) g[q] = Sto<S>::ld(x + (size_t)q * N + e);
    R F[3];
    load_force<S, R>(a.c.force, a.c.Ntot, e, F, D);
    R lfn[Q], lS[NS], lu[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int q = 0; q < Q; ++q) lfn[q] = rec[RL::FN + q];
#pragma unroll
    for (int s = 0; s < NS; ++s) lS[s] = rec[RL::SS + s];
#pragma unroll
    for (int b = 0; b < D; ++b) lu[b] = rec[RL::U + b];
    R lg[Q], lF[3] = {R(0), R(0), R(0)}, lom = R(0);
    post_moments_rev<Q, R>(g, R(a.omega), R(a.c.rho_off), F, rec[RL::RP], lu, lfn, lS, lg, lF, lom);
    add_rows<Q, R>(lam_in, N, e, lg);
    add_force<R>(a.c.lam_force, a.c.Ntot, e, lF, D);
    part[0] += lom;
  }
  store_partials<R, 1>(part, a.c);
}

// ----------------------------------------------------------------- GhostFromCoarser
template <int Q, class S>
__global__ void __launch_bounds__(128) k_adj_gfc(const AdjGfcArgs a) {
  using R = typename Sto<S>::R;
  using LT = Lat<Q>;
  using RL = RecLayout<Q>;
  constexpr int D = LT::D, NS = LT::NS;
  R* __restrict__ lam = static_cast<R*>(a.c.lam_a);
  const R* __restrict__ mom = static_cast<const R*>(a.rec);
  const size_t N = (size_t)a.c.Ntot;
  R part[2] = {R(0), R(0)};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.ng; k += stride) {
    const R* rec[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) rec[s] = mom + (size_t)a.gsrc[(size_t)s * a.ng + k] * RL::STRIDE;
    const uint8_t oct = a.oct[k];
    R sg[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) sg[b] = ((oct >> b) & 1) ? R(1) : R(-1);
    R ul[4][3], Sl[4][NS], rps[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      ul[s][0] = ul[s][1] = ul[s][2] = R(0);
      rps[s] = rec[s][RL::RP];
#pragma unroll
      for (int b = 0; b < D; ++b) ul[s][b] = sg[b] * rec[s][RL::U + b];
#pragma unroll
      for (int b = 0; b < D; ++b)
#pragma unroll
        for (int c = b; c < D; ++c) Sl[s][sidx<D>(b, c)] = sg[b] * sg[c] * rec[s][RL::SS + sidx<D>(b, c)];
    }
    R uloc[3];
    compact_uloc<Q, R>(ul, Sl, uloc);
    R u[3] = {R(0), R(0), R(0)}, usq = R(0);
#pragma unroll
    for (int b = 0; b < D; ++b) {
      u[b] = sg[b] * uloc[b];
      usq += u[b] * u[b];
    }
    const R lw[4] = {D == 3 ? R(0.625) : R(0.5625), D == 3 ? R(0.125) : R(0.1875), D == 3 ? R(0.125) : R(0.1875),
                     D == 3 ? R(0.125) : R(0.0625)};
    const R rp = lw[0] * rps[0] + lw[1] * rps[1] + lw[2] * rps[2] + lw[3] * rps[3];
    const R rho = R(a.c.rho_off) + rp;
    const R wf = R(a.omega_f), wc = R(a.omega_c);
    const R scale = (R(1) - wf) * wc / (R(2) * wf);
    const int64_t e = a.dest0 + k;
    // all loads before the ghost's adjoint is zeroed, so that they overlap
    R lo[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) lo[q] = lam[(size_t)q * N + e];
    R lam_scale = R(0);
#pragma unroll
    for (int q0 = 0; q0 < Q; q0 += 4) {
      R f[4][4];
#pragma unroll
      for (int s = 0; s < 4; ++s) ld4(rec[s] + RL::FN + q0, f[s]);
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (q0 + t < Q) lam_scale += lo[q0 + t] * (lw[0] * f[0][t] + lw[1] * f[1][t] + lw[2] * f[2][t] + lw[3] * f[3][t]);
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) lam[(size_t)q * N + e] = R(0);
    part[0] += lam_scale * (R(1) - wf) / (R(2) * wf);  // d scale / d omega_c
    part[1] += lam_scale * (-wc / (R(2) * wf * wf));    // d scale / d omega_f
    R lam_rp = R(0), lam_u[3] = {R(0), R(0), R(0)};
    geq_rev<Q, R>(lo, rho, u, usq, lam_rp, lam_u);
    R lam_uloc[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int b = 0; b < D; ++b) lam_uloc[b] = sg[b] * lam_u[b];
    // transpose of the linear compact map: column m of its Jacobian by
    // evaluating it on the m-th unit input
    R lul[4][3], lSl[4][NS];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        R eu[4][3] = {}, eS[4][NS] = {}, o[3];
        eu[s][b] = R(1);
        compact_uloc<Q, R>(eu, eS, o);
        lul[s][b] = o[0] * lam_uloc[0] + o[1] * lam_uloc[1] + o[2] * lam_uloc[2];
      }
#pragma unroll
      for (int c = 0; c < NS; ++c) {
        R eu[4][3] = {}, eS[4][NS] = {}, o[3];
        eS[s][c] = R(1);
        compact_uloc<Q, R>(eu, eS, o);
        lSl[s][c] = o[0] * lam_uloc[0] + o[1] * lam_uloc[1] + o[2] * lam_uloc[2];
      }
    }
    R* __restrict__ out = static_cast<R*>(a.contrib) + (size_t)k * 4 * RL::STRIDE;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      R v[RL::STRIDE];
#pragma unroll
      for (int f = 0; f < RL::STRIDE; ++f) v[f] = R(0);
#pragma unroll
      for (int q = 0; q < Q; ++q) v[RL::FN + q] = lw[s] * scale * lo[q];
      v[RL::RP] = lw[s] * lam_rp;
#pragma unroll
      for (int b = 0; b < D; ++b) v[RL::U + b] = sg[b] * lul[s][b];
#pragma unroll
      for (int b = 0; b < D; ++b)
#pragma unroll
        for (int c = b; c < D; ++c) v[RL::SS + sidx<D>(b, c)] = sg[b] * sg[c] * lSl[s][sidx<D>(b, c)];
#pragma unroll
      for (int f = 0; f < RL::STRIDE; f += 4) st4(out + s * RL::STRIDE + f, v + f);
    }
  }
  store_partials<R, 2>(part, a.c);
}

template <class R, int MS>
__global__ void __launch_bounds__(128) k_adj_gather(const AdjGatherArgs a) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.nsrc) return;
  const R* c = static_cast<const R*>(a.contrib);
  R acc[MS];
  R* lr = static_cast<R*>(a.lam_rec) + (size_t)k * MS;
#pragma unroll
  for (int f = 0; f < MS; ++f) acc[f] = lr[f];
  for (int j = a.off[k]; j < a.off[k + 1]; ++j) {
    const R* p = c + (size_t)a.item[j] * MS;
#pragma unroll
    for (int f = 0; f < MS; f += 4) {
      R v[4];
      ld4(p + f, v);
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[f + t] += v[t];
    }
  }
#pragma unroll
  for (int f = 0; f < MS; f += 4) st4(lr + f, acc + f);
}

// ----------------------------------------------------------------- GhostFromFiner
template <int Q, class S>
__global__ void __launch_bounds__(256, LBM_ADJ_MINB(S, LBM_ADJ_GFF_MINB, 1)) k_adj_gff(const AdjGffArgs a) {
  using R = typename Sto<S>::R;
  using LT = Lat<Q>;
  constexpr int D = LT::D, NS = LT::NS, NCH = 1 << D;
  const S* __restrict__ x = static_cast<const S*>(a.c.fsrc);
  // coarse ghosts and fine children: disjoint slots, possibly of one buffer
  R* __restrict__ lam_c = static_cast<R*>(a.c.lam_a);
  R* __restrict__ lam_f = static_cast<R*>(a.c.lam_b);
  const size_t N = (size_t)a.c.Ntot;
  const R wf = R(a.omega_f), wc = R(a.omega_c), rho_off = R(a.c.rho_off);
  R part[2] = {R(0), R(0)};
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  // every lane of a warp runs the same number of iterations (the shuffles need the whole warp)
  const int64_t total = (a.ng * NCH + 31) / 32 * 32;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t - threadIdx.x % 32 < total; t += gstride) {
    const int64_t k = t / NCH;
    const int b = (int)(t % NCH);
    const bool active = k < a.ng;
    R g[Q], F[3] = {R(0), R(0), R(0)};
    R rp = R(0), u[3] = {R(0), R(0), R(0)}, fneq[Q], Sv[NS];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      g[q] = R(0);
      fneq[q] = R(0);
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) Sv[s] = R(0);
    int64_t ec = 0;
    if (active) {
      ec = (int64_t)a.child0[k] + b;
#pragma unroll
      for (int q = 0; q < Q; ++q) g[q] = Sto<S>::ld(x + (size_t)q * N + ec);
      load_force<S, R>(a.c.force, a.c.Ntot, ec, F, D);
      post_moments<Q, R, true>(g, wf, rho_off, F, rp, u, fneq, Sv);
    }
    R dS[3][NS];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const R sgn = ((b >> c) & 1) ? R(1) : R(-1);
#pragma unroll
      for (int s = 0; s < NS; ++s) dS[c][s] = sgn * Sv[s];
    }
    R RP = rp, U[3] = {u[0], u[1], u[2]}, FN[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) FN[q] = fneq[q];
#pragma unroll
    for (int o = 1; o < NCH; o <<= 1) {
      RP += __shfl_xor_sync(0xffffffffu, RP, o);
#pragma unroll
      for (int c = 0; c < D; ++c) U[c] += __shfl_xor_sync(0xffffffffu, U[c], o);
#pragma unroll
      for (int q = 0; q < Q; ++q) FN[q] += __shfl_xor_sync(0xffffffffu, FN[q], o);
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int s = 0; s < NS; ++s) dS[c][s] += __shfl_xor_sync(0xffffffffu, dS[c][s], o);
    }
    // adjoint of the ghost's pdfs: every lane of the group reads all of them,
    // then (after the warp barrier) each lane clears its share of the slots
    const int64_t kk = active ? k : 0;
    const int64_t eg = kk < a.n_inner ? a.dest0 + kk : a.dest_outer + (kk - a.n_inner);
    R lo[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) lo[q] = active ? lam_c[(size_t)q * N + eg] : R(0);
    __syncwarp();
    if (active) {
#pragma unroll
      for (int q = 0; q < Q; ++q)
        if (q % NCH == b) lam_c[(size_t)q * N + eg] = R(0);
    }
    if (!active) continue;
    const R inv = R(1) / R(NCH);
    const R dfac = R(2) * R(D == 3 ? 0.5 : 1.0);
    const R rpm = RP * inv;
    R uP[3] = {R(0), R(0), R(0)}, usq = R(0);
#pragma unroll
    for (int aa = 0; aa < D; ++aa) {
      R lap = R(0);
#pragma unroll
      for (int c = 0; c < D; ++c) lap += dfac * (R(2) * dS[c][sidx<D>(aa, c)] - dS[aa][sidx<D>(c, c)]);
      uP[aa] = U[aa] * inv - lap * R(1.0 / 32.0);
      usq += uP[aa] * uP[aa];
    }
    const R rho = rho_off + rpm;
    const R scale = (R(1) - wc) * R(2) * wf / wc * inv;
    R lam_scale = R(0);
#pragma unroll
    for (int q = 0; q < Q; ++q) lam_scale += lo[q] * FN[q];
    if (b == 0) {
      part[0] += lam_scale * (R(2) * wf * inv) * (-R(1) / (wc * wc));  // d scale / d omega_c
      part[1] += lam_scale * (R(1) - wc) * R(2) / wc * inv;            // d scale / d omega_f
    }
    R lam_rpm = R(0), lam_uP[3] = {R(0), R(0), R(0)};
    geq_rev<Q, R>(lo, rho, uP, usq, lam_rpm, lam_uP);
    R ldS[3][NS];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int s = 0; s < NS; ++s) ldS[c][s] = R(0);
#pragma unroll
    for (int aa = 0; aa < D; ++aa) {
      const R lap_l = -lam_uP[aa] * R(1.0 / 32.0);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        ldS[c][sidx<D>(aa, c)] += dfac * R(2) * lap_l;
        ldS[aa][sidx<D>(c, c)] -= dfac * lap_l;
      }
    }
    // this lane's child
    R lS[NS], lu[3] = {R(0), R(0), R(0)}, lfn[Q];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      R v = R(0);
#pragma unroll
      for (int c = 0; c < D; ++c) v += (((b >> c) & 1) ? R(1) : R(-1)) * ldS[c][s];
      lS[s] = v;
    }
#pragma unroll
    for (int aa = 0; aa < D; ++aa) lu[aa] = lam_uP[aa] * inv;
#pragma unroll
    for (int q = 0; q < Q; ++q) lfn[q] = scale * lo[q];
    R lg[Q], lF[3] = {R(0), R(0), R(0)}, lom = R(0);
    post_moments_rev<Q, R>(g, wf, rho_off, F, lam_rpm * inv, lu, lfn, lS, lg, lF, lom);
    add_rows<Q, R>(lam_f, N, ec, lg);
    add_force<R>(a.c.lam_force, a.c.Ntot, ec, lF, D);
    part[1] += lom;
  }
  store_partials<R, 2>(part, a.c);
}

// ----------------------------------------------------------------- launchers
inline unsigned adj_grid(int64_t n, int threads) {
  const int64_t b = (n + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : (b > kAdjBlocks ? kAdjBlocks : b));
}

template <class S>
struct AdjLaunch {
  static void seed(int Q, const AdjSeedArgs& a, cudaStream_t st) {
    const int64_t n = a.objective == 0 ? a.end - a.begin : a.obs_n;
    with_q(Q, [&](auto q) { k_adj_seed<decltype(q)::value, S><<<adj_grid(n, 256), 256, 0, st>>>(a); });
  }
  static void sc(int Q, const AdjSCArgs& a, cudaStream_t st) {
    with_q(Q, [&](auto q) { k_adj_sc<decltype(q)::value, S><<<kAdjBlocks, 256, 0, st>>>(a); });
  }
  static void sc_brick(int Q, const AdjSCArgs& a, cudaStream_t st) {
    if (a.nB <= 0) return;
    const unsigned g = (unsigned)((a.nB + LBM_BRICKS_PER_BLOCK - 1) / LBM_BRICKS_PER_BLOCK);
    with_q(Q, [&](auto q) { k_adj_sc_brick<decltype(q)::value, S><<<g, LBM_BR_BLOCK, 0, st>>>(a); });
  }
  static void outlet(int Q, const AdjOutletArgs& a, cudaStream_t st) {
    // the normal-link pass writes one row of omega partials per block, so it
    // runs on the full kAdjBlocks grid that k_accum sums over
    if (a.which != 0 && a.end <= a.begin) return;
    const unsigned g = a.which == 0 ? (unsigned)kAdjBlocks : adj_grid(a.end - a.begin, 256);
    with_q(Q, [&](auto q) { k_adj_outlet<decltype(q)::value, S><<<g, 256, 0, st>>>(a); });
  }
  static void moments(int Q, const AdjMomArgs& a, cudaStream_t st) {
    with_q(Q, [&](auto q) { k_adj_moments<decltype(q)::value, S><<<kAdjBlocks, 128, 0, st>>>(a); });
  }
  static void gfc(int Q, const AdjGfcArgs& a, cudaStream_t st) {
    with_q(Q, [&](auto q) { k_adj_gfc<decltype(q)::value, S><<<kAdjBlocks, 128, 0, st>>>(a); });
  }
  static void gff(int Q, const AdjGffArgs& a, cudaStream_t st) {
    with_q(Q, [&](auto q) { k_adj_gff<decltype(q)::value, S><<<kAdjBlocks, 256, 0, st>>>(a); });
  }
};

template <class S>
const AdjOps* make_adj_ops() {
  static const AdjOps ops = {&AdjLaunch<S>::seed,    &AdjLaunch<S>::sc,  &AdjLaunch<S>::sc_brick,
                             &AdjLaunch<S>::outlet,  &AdjLaunch<S>::moments, &AdjLaunch<S>::gfc,
                             &AdjLaunch<S>::gff,     sizeof(typename Sto<S>::R)};
  return &ops;
}

}  // namespace dev
}  // namespace lbm
