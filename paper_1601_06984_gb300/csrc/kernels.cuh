// Device kernels of the multilevel lattice Boltzmann hot path (sm_103a).
//
// Storage S is double (LBM_FP64), float or bfloat16 (deviation storage
// g_i = f_i - w_i rho0, arithmetic in float).  Every kernel is written in the
// deviation form with an offset rho_off (0 for FP64, rho0 otherwise):
//   rho = rho_off + sum g,  g^eq_i = w_i [ (rho - rho_off) + rho (3 c.u + 9/2 (c.u)^2 - 3/2 u.u) ],
// which is Eq. (feq) of Sec. 2.1 minus w_i rho_off.
//
// Memory layout: pdfs A, B as [Q][Ntot] structure-of-arrays over all levels
// (each level a contiguous, padded index range); pull neighbour indices
// nbr[Q-1][Ntot] (uint32, see lbm_internal.h).  One thread per element; the
// direction loops are fully unrolled so every load/store of a warp touches 32
// consecutive elements of one direction array (coalesced), except the pull
// gathers, whose locality comes from the z-curve order.
#pragma once

#include <cuda_bf16.h>
#include <type_traits>
#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {
namespace dev {

// ----------------------------------------------------------------- lattices
template <int Q>
struct Lat;

template <>
struct Lat<9> {
  static constexpr int D = 2, NS = 3;
  __host__ __device__ static constexpr int c(int i, int a) {
    return a == 0   ? ((i == 1 || i == 5 || i == 7) ? 1 : (i == 2 || i == 6 || i == 8) ? -1 : 0)
           : a == 1 ? ((i == 3 || i == 5 || i == 8) ? 1 : (i == 4 || i == 6 || i == 7) ? -1 : 0)
                    : 0;
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
};

template <>
struct Lat<19> {
  static constexpr int D = 3, NS = 6;
  __host__ __device__ static constexpr int c(int i, int a) {
    return a == 0   ? ((i == 1 || i == 7 || i == 9 || i == 11 || i == 13)    ? 1
                       : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1
                                                                               : 0)
           : a == 1 ? ((i == 3 || i == 7 || i == 10 || i == 15 || i == 17)   ? 1
                       : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18)  ? -1
                                                                               : 0)
                    : ((i == 5 || i == 11 || i == 14 || i == 15 || i == 18)  ? 1
                       : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1
                                                                                : 0);
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
};

template <>
struct Lat<27> {
  static constexpr int D = 3, NS = 6;
  // base-3 code (cx+1) + 3 (cy+1) + 9 (cz+1) of each velocity, in lbm.h order
  __host__ __device__ static constexpr int code(int i) {
    return i == 0 ? 13 : i == 1 ? 14 : i == 2 ? 12 : i == 3 ? 16 : i == 4 ? 10 : i == 5 ? 22 : i == 6 ? 4 : i == 7 ? 17 : i == 8 ? 9 : i == 9 ? 11 : i == 10 ? 15 : i == 11 ? 23 : i == 12 ? 3 : i == 13 ? 5 : i == 14 ? 21 : i == 15 ? 25 : i == 16 ? 1 : i == 17 ? 7 : i == 18 ? 19 : i == 19 ? 26 : i == 20 ? 0 : i == 21 ? 8 : i == 22 ? 18 : i == 23 ? 20 : i == 24 ? 6 : i == 25 ? 24 : 2;
  }
  __host__ __device__ static constexpr int c(int i, int a) {
    return (a == 0 ? code(i) % 3 : (a == 1 ? code(i) / 3 % 3 : code(i) / 9)) - 1;
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 8.0 / 27.0 : (i <= 6 ? 2.0 / 27.0 : (i <= 18 ? 1.0 / 54.0 : 1.0 / 216.0));
  }
};

__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// Run-time lookup of c_{i,a} and w_i for a velocity index known only at run
// time (a lane's share of the directions): c_{i,a} + 1 packed in two bits per
// velocity; the weights depend on |c_i|^2, i.e. on the index range (every
// lattice lists its velocities by increasing length).
template <int Q>
struct LatRt {
  __host__ __device__ static constexpr uint64_t pack(int a) {
    uint64_t m = 0;
    for (int i = 0; i < Q; ++i) m |= (uint64_t)(Lat<Q>::c(i, a) + 1) << (2 * i);
    return m;
  }
  __device__ static __forceinline__ int c(int i, int a) {
    constexpr uint64_t X = pack(0), Y = pack(1), Z = pack(2);
    const uint64_t m = a == 0 ? X : (a == 1 ? Y : Z);
    return (int)((m >> (2 * i)) & 3u) - 1;
  }
  template <class R>
  __device__ static __forceinline__ R w(int i) {
    constexpr int D = Lat<Q>::D;
    return i == 0 ? R(Lat<Q>::w(0))
                  : (i <= 2 * D ? R(Lat<Q>::w(1)) : ((Q == 27 && i > 18) ? R(Lat<Q>::w(19)) : R(Lat<Q>::w(2 * D + 1))));
  }
};

// index of S_ab in the packed strain-rate vector (xx,yy,xy | xx,yy,zz,xy,yz,xz)
template <int D>
__host__ __device__ constexpr int sidx(int a, int b) {
  return a == b ? a
                : (D == 2 ? 2
                          : ((a + b == 1) ? 3 : ((a + b == 3) ? 4 : 5)));
}

// ----------------------------------------------------------------- storage
template <class S>
struct Sto;
template <>
struct Sto<double> {
  using R = double;
  __device__ static __forceinline__ R ld(const double* p) { return *p; }
  __device__ static __forceinline__ double cv(R v) { return v; }
};
template <>
struct Sto<float> {
  using R = float;
  __device__ static __forceinline__ R ld(const float* p) { return *p; }
  __device__ static __forceinline__ float cv(R v) { return v; }
};
template <>
struct Sto<__nv_bfloat16> {
  using R = float;
  __device__ static __forceinline__ R ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  __device__ static __forceinline__ __nv_bfloat16 cv(R v) { return __float2bfloat16_rn(v); }
};

// ----------------------------------------------------------------- physics
// g^eq_i for density deviation rp = rho - rho_off
template <int Q, class R>
__device__ __forceinline__ R geq(int i, R rp, R rho, const R* u, R usq) {
  using LT = Lat<Q>;
  R cu = R(0);
#pragma unroll
  for (int a = 0; a < LT::D; ++a) cu += R(LT::c(i, a)) * u[a];
  return R(LT::w(i)) * (rp + rho * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq));
}

// Guo forcing term (1 - omega/2) w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F
template <int Q, class R>
__device__ __forceinline__ R guo(int i, R omega, const R* u, const R* F) {
  using LT = Lat<Q>;
  R cu = R(0), cF = R(0), uF = R(0);
#pragma unroll
  for (int a = 0; a < LT::D; ++a) {
    cu += R(LT::c(i, a)) * u[a];
    cF += R(LT::c(i, a)) * F[a];
    uF += u[a] * F[a];
  }
  return (R(1) - R(0.5) * omega) * R(LT::w(i)) * (R(3) * (cF - uF) + R(9) * cu * cF);
}

// rho deviation and first moment of a pdf set
template <int Q, class R>
__device__ __forceinline__ void raw_moments(const R* g, R& rp, R* j) {
  using LT = Lat<Q>;
  rp = R(0);
  j[0] = j[1] = j[2] = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    rp += g[i];
#pragma unroll
    for (int a = 0; a < LT::D; ++a) {
      if (LT::c(i, a) > 0) j[a] += g[i];
      if (LT::c(i, a) < 0) j[a] -= g[i];
    }
  }
}

// Pre-collision moments from a stored post-collision set: u = (j - F/2)/rho,
// f^neq = (g - g^eq - F_i) / (1 - omega), S_ab = -(3 omega / 2 rho) sum c_a c_b f^neq.
// g^eq per pair of opposite velocities (c.u changes sign: the even part is
// shared); without FORCE the forcing terms are left out at compile time.
template <int Q, class R, bool WANT_S, bool FORCE = true>
__device__ __forceinline__ void post_moments(const R* g, R omega, R rho_off, const R* F, R& rp, R* u,
                                             R* fneq, R* S) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  R j[3];
  raw_moments<Q, R>(g, rp, j);
  const R rho = rho_off + rp;
  const R inv = R(1) / rho;
  u[0] = u[1] = u[2] = R(0);
#pragma unroll
  for (int a = 0; a < D; ++a) u[a] = (FORCE ? j[a] - R(0.5) * F[a] : j[a]) * inv;
  R usq = R(0);
#pragma unroll
  for (int a = 0; a < D; ++a) usq += u[a] * u[a];
  const R r1w = R(1) / (R(1) - omega);
  const R base = rp - R(1.5) * rho * usq;
  {
    R f0 = g[0] - R(LT::w(0)) * base;
    if (FORCE) f0 -= guo<Q, R>(0, omega, u, F);
    fneq[0] = f0 * r1w;
  }
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    R cu = R(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      if (LT::c(i, a) > 0) cu += u[a];
      if (LT::c(i, a) < 0) cu -= u[a];
    }
    const R w = R(LT::w(i));
    const R even = w * (base + R(4.5) * rho * cu * cu);
    const R odd = w * R(3) * rho * cu;
    R fa = g[i] - (even + odd), fb = g[i + 1] - (even - odd);
    if (FORCE) {
      fa -= guo<Q, R>(i, omega, u, F);
      fb -= guo<Q, R>(i + 1, omega, u, F);
    }
    fneq[i] = fa * r1w;
    fneq[i + 1] = fb * r1w;
  }
  if (WANT_S) {
    const R pre = -R(1.5) * omega * inv;
#pragma unroll
    for (int s = 0; s < LT::NS; ++s) S[s] = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b) {
          const int cc = LT::c(i, a) * LT::c(i, b);
          if (cc > 0) S[sidx<D>(a, b)] += fneq[i];
          if (cc < 0) S[sidx<D>(a, b)] -= fneq[i];
        }
    }
#pragma unroll
    for (int s = 0; s < LT::NS; ++s) S[s] *= pre;
  }
}

// ----------------------------------------------------------------- GFC source records
// Record of one source (compute type, mom_stride(Q) values, 16-byte aligned
// groups): f^neq[Q] padded to a multiple of 4, then rho - rho_off, u[D], S[nS],
// padding.  Vector loads/stores move a record in 8 (float) or 16 (double) pieces.
template <int Q>
struct RecLayout {
  static constexpr int D = Lat<Q>::D, NS = Lat<Q>::NS;
  static constexpr int FN = 0;
  static constexpr int RP = (Q + 3) / 4 * 4;
  static constexpr int U = RP + 1;
  static constexpr int SS = U + D;
  static constexpr int END = SS + NS;
  static constexpr int STRIDE = mom_stride(Q);
  static_assert(END <= STRIDE && STRIDE % 4 == 0, "moment record too long");
};

__device__ __forceinline__ void ld4(const float* p, float* o) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double* o) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  o[0] = a.x;
  o[1] = a.y;
  o[2] = b.x;
  o[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double* v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// Interpolation step 1 (Sec. 2.2) for one source: its record from its stored
// (post-collision) pdfs g.
template <int Q, class R, bool FORCE>
__device__ __forceinline__ void source_record(const R (&g)[Q], R omega, R rho_off, const R* F,
                                              R (&rec)[RecLayout<Q>::STRIDE]) {
  using RL = RecLayout<Q>;
  constexpr int D = Lat<Q>::D, NS = Lat<Q>::NS;
#pragma unroll
  for (int f = 0; f < RL::STRIDE; ++f) rec[f] = R(0);
  R rp, u[3], fneq[Q], Sv[NS];
  post_moments<Q, R, true, FORCE>(g, omega, rho_off, F, rp, u, fneq, Sv);
#pragma unroll
  for (int q = 0; q < Q; ++q) rec[RL::FN + q] = fneq[q];
  rec[RL::RP] = rp;
#pragma unroll
  for (int b = 0; b < D; ++b) rec[RL::U + b] = u[b];
#pragma unroll
  for (int s = 0; s < NS; ++s) rec[RL::SS + s] = Sv[s];
}

// rec := (prev + rec) / 2; the whole previous record is read before the
// caller's first store (the compiler cannot tell the records apart and would
// otherwise serialise loads and stores)
template <int Q, class R>
__device__ __forceinline__ void mean_record(const R* __restrict__ prev, R (&rec)[RecLayout<Q>::STRIDE]) {
  using RL = RecLayout<Q>;
  R pv[RL::STRIDE];
#pragma unroll
  for (int f = 0; f < RL::END; f += 4) ld4(prev + f, pv + f);
#pragma unroll
  for (int f = 0; f < RL::END; ++f) rec[f] = R(0.5) * (pv[f] + rec[f]);
}

template <int Q, class R>
__device__ __forceinline__ void store_record(R* __restrict__ out, const R (&rec)[RecLayout<Q>::STRIDE]) {
#pragma unroll
  for (int f = 0; f < RecLayout<Q>::END; f += 4) st4(out + f, rec + f);
}

// Stream-collide epilogue for a GhostFromCoarser source among the processed
// elements: g are the element's new values before rounding to storage; the
// record is taken from the values as stored, so it equals what
// k_source_moments computes from the stored state.  Mask words are per 32
// slots: one broadcast load for a warp of consecutive elements.
template <int Q, class S, bool FORCE>
__device__ __forceinline__ void source_out(const SourceOut& so, int64_t e, const typename Sto<S>::R (&g)[Q],
                                           typename Sto<S>::R omega, typename Sto<S>::R rho_off,
                                           const typename Sto<S>::R* F) {
  using R = typename Sto<S>::R;
  using RL = RecLayout<Q>;
  const uint32_t m = __ldg(so.mask + (e >> 5));
  const uint32_t bit = (uint32_t)e & 31u;
  if (!((m >> bit) & 1u)) return;
  const int64_t k = (int64_t)__ldg(so.first + (e >> 5)) + __popc(m & ((1u << bit) - 1u));
  R gs[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const S v = Sto<S>::cv(g[q]);
    gs[q] = Sto<S>::ld(&v);
  }
  R rec[RL::STRIDE];
  source_record<Q, R, FORCE>(gs, omega, rho_off, F, rec);
  store_record<Q, R>(static_cast<R*>(so.rec_out) + k * RL::STRIDE, rec);
}

// ----------------------------------------------------------------- stream + collide
// Tuning knobs of the hot kernel (compile-time; the defaults are the measured
// best on GB300).  LBM_SC_EPT: elements per thread; LBM_SC_BLOCK: threads per
// block; LBM_SC_MINB: minimum resident blocks per SM for __launch_bounds__;
// LBM_SC_STREAM: streaming (evict-first) hints on the use-once neighbour
// indices and on the stores.
#ifndef LBM_SC_EPT
#define LBM_SC_EPT 1
#endif
#ifndef LBM_SC_BLOCK
#define LBM_SC_BLOCK 256
#endif
#ifndef LBM_SC_MINB
#define LBM_SC_MINB 4
#endif
#ifndef LBM_SC_STREAM
#define LBM_SC_STREAM 1
#endif

__device__ __forceinline__ uint32_t ld_once(const uint32_t* p) {
#if LBM_SC_STREAM
  return __ldcs(p);
#else
  return __ldg(p);
#endif
}
__device__ __forceinline__ void st_once(double* p, double v) {
#if LBM_SC_STREAM
  __stcs(p, v);
#else
  *p = v;
#endif
}
__device__ __forceinline__ void st_once(float* p, float v) {
#if LBM_SC_STREAM
  __stcs(p, v);
#else
  *p = v;
#endif
}
__device__ __forceinline__ void st_once(__nv_bfloat16* p, __nv_bfloat16 v) {
#if LBM_SC_STREAM
  __stcs(reinterpret_cast<unsigned short*>(p), __bfloat16_as_ushort(v));
#else
  *p = v;
#endif
}

// BGK collision (Eq. bgk) of one element in place, with Guo forcing, using the
// symmetry of each velocity pair (i, opp(i)): c.u and c.F change sign, so the
// even part of f^eq (and of the forcing term) is shared and the odd part flips.
template <int Q, class R, bool FORCE>
__device__ __forceinline__ void bgk_collide(R (&g)[Q], R om, R rho_off, const R* F) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  R rp, j[3];
  raw_moments<Q, R>(g, rp, j);
  const R rho = rho_off + rp;
  const R inv = R(1) / rho;
  R u[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int b = 0; b < D; ++b) u[b] = (j[b] + (FORCE ? R(0.5) * F[b] : R(0))) * inv;
  R usq = R(0), uF = R(0);
#pragma unroll
  for (int b = 0; b < D; ++b) {
    usq += u[b] * u[b];
    if (FORCE) uF += u[b] * F[b];
  }
  const R base = rp - R(1.5) * rho * usq;  // even part without the (c.u)^2 term, per unit weight
  const R fpre = FORCE ? (R(1) - R(0.5) * om) : R(0);
  {
    R geq0 = R(LT::w(0)) * base;
    R gi = g[0] + om * (geq0 - g[0]);
    if (FORCE) gi += fpre * R(LT::w(0)) * (-R(3) * uF);
    g[0] = gi;
  }
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    R cu = R(0), cF = R(0);
#pragma unroll
    for (int b = 0; b < D; ++b) {
      if (LT::c(i, b) > 0) {
        cu += u[b];
        if (FORCE) cF += F[b];
      }
      if (LT::c(i, b) < 0) {
        cu -= u[b];
        if (FORCE) cF -= F[b];
      }
    }
    const R w = R(LT::w(i));
    const R even = w * (base + R(4.5) * rho * cu * cu);
    const R odd = w * R(3) * rho * cu;
    R a = g[i] + om * (even + odd - g[i]);
    R b = g[i + 1] + om * (even - odd - g[i + 1]);
    if (FORCE) {
      const R fe = fpre * w * (R(9) * cu * cF - R(3) * uF);
      const R fo = fpre * w * R(3) * cF;
      a += fe + fo;
      b += fe - fo;
    }
    g[i] = a;
    g[i + 1] = b;
  }
}

// Pull streaming f_i(x) = f*_i(x - c_i) through the neighbour list (Sec. 2.1,
// Eq. lbe) fused with the BGK collision (Eq. bgk).  Every thread first issues
// all neighbour-index loads, then all pdf gathers (branch-free: codes other than
// a plain pull read the element's own opposite slot, which is the bounce-back
// value), and patches the rare inlet / outlet values afterwards, so that up to
// 2(Q-1) independent loads per element are in flight.
template <int Q, class S, bool FORCE, int EPT, bool MOMS>
__global__ void __launch_bounds__(LBM_SC_BLOCK, LBM_SC_MINB) k_stream_collide(const StreamCollideArgs a) {
  using R = typename Sto<S>::R;
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  const int64_t l0 = a.begin + (int64_t)blockIdx.x * (LBM_SC_BLOCK * EPT) + threadIdx.x;
  const S* __restrict__ src = static_cast<const S*>(a.src);
  S* __restrict__ dst = static_cast<S*>(a.dst);
  const uint32_t* __restrict__ nbr = a.nbr;
  const size_t N = (size_t)a.Ntot;
  // linear position -> element, stepping over the interior bricks; linear
  // positions at or past a.end are idle
  int64_t el[EPT];
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int64_t lin = l0 + k * LBM_SC_BLOCK;
    el[k] = lin >= a.end ? -1 : lin + (lin >= a.hole_at ? a.hole_len : 0);
  }
  uint32_t nb[EPT][Q - 1];
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int64_t e = el[k];
    if (e >= 0) {
#pragma unroll
      for (int i = 1; i < Q; ++i) nb[k][i - 1] = ld_once(nbr + (size_t)(i - 1) * N + e);
    }
  }
  R g[EPT][Q];
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int64_t e = el[k];
    if (e >= 0) {
      g[k][0] = Sto<S>::ld(src + e);
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const uint32_t n = nb[k][i - 1];
        const size_t idx = n < NB_FLAG30 ? (size_t)i * N + n : (size_t)opp(i) * N + (size_t)e;
        g[k][i] = Sto<S>::ld(src + idx);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int64_t e = el[k];
    if (e < 0) continue;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t n = nb[k][i - 1];
      if (n >= NB_FLAG30) {
        if (n & NB_BOUNCE) {
          if (n & NB_FLAG30) g[k][i] += R(a.inlet[i]) * (a.inlet_s ? R(a.inlet_s[n & NB_INDEX]) : R(1));
        } else {
          g[k][i] = static_cast<const R*>(a.side)[n & NB_INDEX];
        }
      }
    }
    R F[3] = {R(0), R(0), R(0)};
    if (FORCE) {
      const R* __restrict__ fp = static_cast<const R*>(a.force);
#pragma unroll
      for (int b = 0; b < D; ++b) F[b] = fp[(size_t)b * N + e];
    }
    bgk_collide<Q, R, FORCE>(g[k], R(a.omega), R(a.rho_off), F);
#pragma unroll
    for (int i = 0; i < Q; ++i) st_once(dst + (size_t)i * N + e, Sto<S>::cv(g[k][i]));
    if (MOMS) source_out<Q, S, FORCE>(a.so, e, g[k], R(a.omega), R(a.rho_off), F);
  }
}

// Stream-collide of interior bricks: the same pull and BGK collision as
// k_stream_collide, with the pull source of link i located by the brick's
// neighbour row instead of the per-element neighbour list.  Each group of 64
// threads takes one brick, thread l its element at z-curve position l; blocks
// are issued in brick order, so the bricks in flight stay a compact window of
// the level and their neighbours' lines are still in L2 when gathered.  The
// thread's Q-1 link-table entries (slot, position) are loaded into registers,
// lanes 0..26 of each warp load the brick's 27-entry neighbour row in one
// coalesced access, and every link takes its row entry by a warp shuffle, so
// all pdf gathers issue after two loads.  The element's HBM traffic is its Q
// pdf reads and Q writes.
#ifndef LBM_BR_BLOCK
#define LBM_BR_BLOCK 256
#endif
#ifndef LBM_BR_MINB
#define LBM_BR_MINB 4
#endif
//
// Boundary bricks (BND): a complete brick whose neighbour brick behind some
// link is not complete; those links (row entry kBrickMissing) take the
// element's neighbour-list code like k_stream_collide: a pull, the element's
// own opposite slot (bounce-back), plus the inlet term, or a boundary value.
// Every link is first resolved to one 32-bit offset, so the gathers need no
// branch.  Five blocks per SM (48 registers, no spills) for D3Q19 and D2Q9
// with 4-byte or narrower storage (measured: 4.66 against 4.38 TB/s at four);
// three where more registers are needed (D3Q27, FP64).
#ifndef LBM_BR_BND_MINB_NARROW
#define LBM_BR_BND_MINB_NARROW 5
#endif
#define LBM_BR_BND_MINB(Q, S) ((Q) > 19 || sizeof(S) > 4 ? 3 : LBM_BR_BND_MINB_NARROW)
// Interior bricks: BF16 storage moves half the bytes per element, so it needs
// more elements in flight; five blocks per SM (48 registers, no spills) for
// D3Q19 / D2Q9 BF16, measured faster than four or six.
#define LBM_BR_INT_MINB(Q, S) ((Q) <= 19 && sizeof(S) == 2 ? 5 : LBM_BR_MINB)
#define LBM_BR_MOMS_MINB(Q, S) ((Q) <= 19 && sizeof(S) <= 4 ? 5 : LBM_BR_MINB)

template <int Q, class S, bool FORCE, bool BND, bool MOMS>
__global__ void __launch_bounds__(LBM_BR_BLOCK, BND ? LBM_BR_BND_MINB(Q, S) : (MOMS ? LBM_BR_MOMS_MINB(Q, S) : LBM_BR_INT_MINB(Q, S))) k_stream_collide_brick(const BrickArgs a) {
  using R = typename Sto<S>::R;
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  constexpr int BPB = LBM_BR_BLOCK / 64;
  constexpr int NW = Q / 2;  // (Q-1)/2 words of two 16-bit entries
  const int l = threadIdx.x & 63, lane = threadIdx.x & 31;
  // the brick index is uniform over each warp (64 threads per brick), so the
  // exit below and the shuffles run with whole warps
  const int64_t b = (int64_t)blockIdx.x * BPB + (threadIdx.x >> 6);
  if (b >= a.nB) return;
  uint32_t tw[NW];
#pragma unroll
  for (int k = 0; k < NW; ++k)
    tw[k] = (uint32_t)__ldg(a.tab + (2 * k) * 64 + l) | ((uint32_t)__ldg(a.tab + (2 * k + 1) * 64 + l) << 16);
  const int32_t row = lane < 27 ? __ldg(a.nb + b * 27 + lane) : 0;
  const size_t N = (size_t)a.Ntot;
  // offsets below are relative to the brick's first element
  const int64_t first = a.begin + b * 64;
  const S* __restrict__ src = static_cast<const S*>(a.src) + first;
  S* __restrict__ dst = static_cast<S*>(a.dst) + first + l;
  R g[Q];
  g[0] = Sto<S>::ld(src + l);
  if (!BND) {
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t v = (tw[(i - 1) >> 1] >> (((i - 1) & 1) * 16)) & 0xffffu;
      const int32_t r = __shfl_sync(0xffffffffu, row, (int)(v >> 6));
      g[i] = Sto<S>::ld(src + (int64_t)(i * N) + r + (v & 63));
    }
  } else {
    // phase 1: every link's pull source as one 32-bit offset from src + i N
    // (src starts at the brick's first element): the brick-table entry, or,
    // through a missing neighbour brick, the element's neighbour-list code
    // resolved to a pull (n - first), to its own opposite slot (bounce-back,
    // and the inlet's base value: (opp(i) - i) N + l), or, for a boundary
    // value, to that same valid slot, the value being substituted below.
    // |offsets| < 2^30 + 64 since Ntot < 2^30.  Links whose value gets an
    // inlet term or a substitute are marked in `patch`.
    const int64_t e = first + l;
    int32_t off[Q];
    uint32_t miss = 0, patch = 0;
    off[0] = 0;
    // 1a: brick-table offsets; the codes of links through missing bricks are
    // loaded, all before any of them is used
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const uint32_t v = (tw[(i - 1) >> 1] >> (((i - 1) & 1) * 16)) & 0xffffu;
      const int32_t r = __shfl_sync(0xffffffffu, row, (int)(v >> 6));
      if (r != kBrickMissing) {
        off[i] = r + (int32_t)(v & 63);
      } else {
        off[i] = (int32_t)__ldg(a.nbr + (size_t)(i - 1) * N + e);
        miss |= 1u << i;
      }
    }
    // 1b: the codes resolved to offsets
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (!((miss >> i) & 1u)) continue;
      const uint32_t n = (uint32_t)off[i];
      if (n < NB_FLAG30) {
        off[i] = (int32_t)((int64_t)n - first);
      } else {
        off[i] = (int32_t)((int64_t)(opp(i) - i) * (int64_t)N + l);
        if (n & NB_FLAG30) patch |= 1u << i;
      }
    }
    // phase 2: the gathers, branch-free
#pragma unroll
    for (int i = 1; i < Q; ++i) g[i] = Sto<S>::ld(src + (int64_t)(i * N) + off[i]);
    // phase 3 (inlet and boundary-value elements only): the inlet term or the
    // precomputed boundary value, from the link's code read again
    if (patch) {
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        if (!((patch >> i) & 1u)) continue;
        const uint32_t n = __ldg(a.nbr + (size_t)(i - 1) * N + e);
        if (n & NB_BOUNCE) g[i] += R(a.inlet[i]) * (a.inlet_s ? R(a.inlet_s[n & NB_INDEX]) : R(1));
        else g[i] = static_cast<const R*>(a.side)[n & NB_INDEX];
      }
    }
  }
  R F[3] = {R(0), R(0), R(0)};
  if (FORCE) {
    const R* __restrict__ fp = static_cast<const R*>(a.force) + first + l;
#pragma unroll
    for (int c = 0; c < D; ++c) F[c] = fp[c * N];
  }
  bgk_collide<Q, R, FORCE>(g, R(a.omega), R(a.rho_off), F);
#pragma unroll
  for (int i = 0; i < Q; ++i) st_once(dst + i * N, Sto<S>::cv(g[i]));
  if (MOMS) source_out<Q, S, FORCE>(a.so, first + l, g, R(a.omega), R(a.rho_off), F);
}

// BF16 interior bricks, two neighbouring elements per thread: lane m of the
// brick's warp takes z-curve positions 2m and 2m+1, which differ only in the
// lowest x bit, so they sit next to each other in every direction array.  A
// link with c_x = 0 pulls both sources from one brick slot at positions l'
// and l'+1 (the mesh builder checks this on the link table), one 32-bit
// bfloat16 pair load at an even element index; links with c_x != 0 take two
// single loads.  The 19 results are written as bfloat16 pairs, rounded by one
// packed conversion each.  Same pull and BGK collision as the one-element
// kernel, element by element.
// 128-thread blocks (four bricks), 1024 threads per SM (64 registers) for
// D2Q9 / D3Q19, 768 for D3Q27 (which spills at 1024).  Measured on the
// sphere's finest level: 5.46 TB/s against 5.37 with 256-thread blocks and
// 4.91 with 512; 1280 threads per SM (48 registers) spilled and was slower.
// plain stores (no evict-first hint) measured 0.3% faster for this kernel
#ifndef LBM_PAIR_STCS
#define LBM_PAIR_STCS 0
#endif
#ifndef LBM_BR_PAIR_BLOCK
#define LBM_BR_PAIR_BLOCK 128
#endif
#ifndef LBM_BR_PAIR_MINB_Q19
#define LBM_BR_PAIR_MINB_Q19 (1024 / LBM_BR_PAIR_BLOCK)
#endif
#define LBM_BR_PAIR_MINB(Q) ((Q) > 19 ? 768 / LBM_BR_PAIR_BLOCK : LBM_BR_PAIR_MINB_Q19)
template <int Q, bool FORCE>
__global__ void __launch_bounds__(LBM_BR_PAIR_BLOCK, LBM_BR_PAIR_MINB(Q)) k_stream_collide_brick_pair(const BrickArgs a) {
  using S = __nv_bfloat16;
  using R = float;
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  constexpr int BPB = LBM_BR_PAIR_BLOCK / 32;
  const int m = threadIdx.x & 31;
  // one brick per warp: the exit below and the shuffles run with whole warps
  const int64_t b = (int64_t)blockIdx.x * BPB + (threadIdx.x >> 5);
  if (b >= a.nB) return;
  const int32_t row = m < 27 ? __ldg(a.nb + b * 27 + m) : 0;
  const size_t N = (size_t)a.Ntot;
  const int64_t first = a.begin + b * 64;
  const S* __restrict__ src = static_cast<const S*>(a.src) + first;
  S* __restrict__ dst = static_cast<S*>(a.dst) + first + 2 * m;
  // the link-table entries of positions 2m (low half) and 2m+1 (high half)
  const uint32_t* __restrict__ tab2 = reinterpret_cast<const uint32_t*>(a.tab);
  R g0[Q], g1[Q];
  {
    const __nv_bfloat162 p = *reinterpret_cast<const __nv_bfloat162*>(src + 2 * m);
    g0[0] = __low2float(p);
    g1[0] = __high2float(p);
  }
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const uint32_t tw = __ldg(tab2 + (i - 1) * 32 + m);
    const S* base = src + (int64_t)(i * N);
    if (LT::c(i, 0) == 0) {
      const uint32_t v = tw & 0xffffu;
      const int32_t r = __shfl_sync(0xffffffffu, row, (int)(v >> 6));
      const __nv_bfloat162 p = *reinterpret_cast<const __nv_bfloat162*>(base + (r + (int32_t)(v & 63)));
      g0[i] = __low2float(p);
      g1[i] = __high2float(p);
    } else {
      const uint32_t v0 = tw & 0xffffu, v1 = tw >> 16;
      const int32_t r0 = __shfl_sync(0xffffffffu, row, (int)(v0 >> 6));
      const int32_t r1 = __shfl_sync(0xffffffffu, row, (int)(v1 >> 6));
      // signed sums: a neighbour brick stored before this one has r < 0
      g0[i] = __bfloat162float(base[r0 + (int32_t)(v0 & 63)]);
      g1[i] = __bfloat162float(base[r1 + (int32_t)(v1 & 63)]);
    }
  }
  R F0[3] = {R(0), R(0), R(0)}, F1[3] = {R(0), R(0), R(0)};
  if (FORCE) {
    const R* __restrict__ fp = static_cast<const R*>(a.force) + first + 2 * m;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const float2 f = *reinterpret_cast<const float2*>(fp + c * N);
      F0[c] = f.x;
      F1[c] = f.y;
    }
  }
  bgk_collide<Q, R, FORCE>(g0, R(a.omega), R(a.rho_off), F0);
  bgk_collide<Q, R, FORCE>(g1, R(a.omega), R(a.rho_off), F1);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(g0[i], g1[i]);
#if LBM_SC_STREAM && LBM_PAIR_STCS
    __stcs(reinterpret_cast<unsigned int*>(dst + i * N), *reinterpret_cast<const unsigned int*>(&p));
#else
    *reinterpret_cast<__nv_bfloat162*>(dst + i * N) = p;
#endif
  }
}

// ----------------------------------------------------------------- outlet values
// Sec. 2.3 outflow: for an incoming direction i whose upstream element lies
// beyond the outlet, either extrapolate that element's f_i linearly along -n
// (2 f_i(x - c_i - n) - f_i(x - c_i - 2n); optionally zero-gradient,
// f_i(x - c_i - n)), or, for c_i = -n, correct the pressure:
// f^eq_i(rho0, u) + f^neq_opp(i)(x) with the pre-collision f^neq.
template <int Q, class S>
__global__ void k_outlet(const OutletArgs a) {
  using R = typename Sto<S>::R;
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  const int64_t k = a.begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.end) return;
  const S* __restrict__ src = static_cast<const S*>(a.src);
  const size_t N = (size_t)a.Ntot;
  const int i = a.dir[k];
  R* side = static_cast<R*>(a.side);
  if (a.kind[k] == OUT_EXTRAP) {
    const R fa = Sto<S>::ld(src + (size_t)i * N + a.a[k]);
    side[k] = a.zero_gradient ? fa : R(2) * fa - Sto<S>::ld(src + (size_t)i * N + a.b[k]);
    return;
  }
  if (a.kind[k] == OUT_BOUZIDI) {
    // interpolated bounce-back with the wall at x - q c_i (Sec. 2.3, Bouzidi):
    //   q <  1/2: 2q f*_ib(x) + (1 - 2q) f*_ib(x + c_i)
    //   q >= 1/2: f*_ib(x) / (2q) + (2q - 1) / (2q) f*_i(x)
    // (deviation storage: the weights of each branch sum to one and w_i = w_ib)
    const int ib = opp(i);
    const int64_t e = a.elem[k];
    const double q = a.q ? a.q[k] : 0.5;
    const R fo = Sto<S>::ld(src + (size_t)ib * N + e);
    if (q < 0.5) {
      const int32_t a2 = a.a[k];
      side[k] = a2 < 0 ? fo : R(2.0 * q) * fo + R(1.0 - 2.0 * q) * Sto<S>::ld(src + (size_t)ib * N + a2);
    } else {
      side[k] = R(1.0 / (2.0 * q)) * fo + R((2.0 * q - 1.0) / (2.0 * q)) * Sto<S>::ld(src + (size_t)i * N + e);
    }
    return;
  }
  const int64_t e = a.elem[k];
  R g[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) g[q] = Sto<S>::ld(src + (size_t)q * N + e);
  R F[3] = {R(0), R(0), R(0)};
  if (a.force)
#pragma unroll
    for (int b = 0; b < D; ++b) F[b] = static_cast<const R*>(a.force)[(size_t)b * N + e];
  R rp, j[3];
  raw_moments<Q, R>(g, rp, j);
  const R rho = R(a.rho_off) + rp;
  R u[3] = {R(0), R(0), R(0)};
  R usq = R(0);
#pragma unroll
  for (int b = 0; b < D; ++b) {
    u[b] = (j[b] - R(0.5) * F[b]) / rho;
    usq += u[b] * u[b];
  }
  const int ib = opp(i);
  R gib = R(0);
#pragma unroll
  for (int q = 0; q < Q; ++q)
    if (q == ib) gib = g[q];
  // f^eq_i(rho0, u) + f^neq_ib, f^neq the pre-collision non-equilibrium part
  // recovered from the stored post-collision pdf: (f* - f^eq - F_ib) / (1 - omega)
  const R om = R(a.omega);
  const R fneq_ib = (gib - geq<Q, R>(ib, rp, rho, u, usq) - guo<Q, R>(ib, om, u, F)) * (R(1) / (R(1) - om));
  const R r0 = R(a.rho0);
  side[k] = geq<Q, R>(i, r0 - R(a.rho_off), r0, u, usq) + fneq_ib;
}

// ----------------------------------------------------------------- GFC source moments
// Interpolation step 1 (Sec. 2.2) as a kernel of its own: density, velocity,
// strain rate and f^neq of the listed sources (elem[k], record rec[k] or k).
// With prev set, the record is the mean of prev and the moments now (the
// source moments at t+1/2 of the linear-in-time mode).  During the steps the
// stream-collide writes the records of the sources it updates (source_out);
// this kernel takes the GhostFromFiner sources after their fill and every
// source when the records have to be rebuilt from a new state.
// Launch bounds of the ghost kernels: LBM_*_MINB sets a minimum of resident
// blocks per SM; unset (0), only the block size is given, which lets the
// compiler use fewer registers than an explicit minimum of one block.
#ifndef LBM_MOM_BLOCK
#define LBM_MOM_BLOCK 128
#endif
#if defined(LBM_MOM_MINB) && LBM_MOM_MINB > 0
#define LBM_MOM_BOUNDS __launch_bounds__(LBM_MOM_BLOCK, LBM_MOM_MINB)
#else
#define LBM_MOM_BOUNDS __launch_bounds__(LBM_MOM_BLOCK)
#endif
template <int Q, class S, bool FORCE>
__global__ void LBM_MOM_BOUNDS k_source_moments(const MomentsArgs a) {
  using R = typename Sto<S>::R;
  using RL = RecLayout<Q>;
  constexpr int D = Lat<Q>::D;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.nsrc) return;
  const S* __restrict__ src = static_cast<const S*>(a.src);
  const size_t N = (size_t)a.Ntot;
  const int64_t e = a.elem[k];
  const int64_t r = a.rec ? (int64_t)a.rec[k] : k;
  R g[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) g[q] = Sto<S>::ld(src + (size_t)q * N + e);
  R F[3] = {R(0), R(0), R(0)};
  if (FORCE)
#pragma unroll
    for (int b = 0; b < D; ++b) F[b] = static_cast<const R*>(a.force)[(size_t)b * N + e];
  R rec[RL::STRIDE];
  source_record<Q, R, FORCE>(g, R(a.omega), R(a.rho_off), F, rec);
  if (a.prev) mean_record<Q, R>(static_cast<const R*>(a.prev) + (size_t)r * RL::STRIDE, rec);
  store_record<Q, R>(static_cast<R*>(a.mom) + (size_t)r * RL::STRIDE, rec);
}

// Compact quadratic velocity at the ghost in the octant's local frame, a linear
// map of the sources' local-frame velocities ul and strain rates Sl (see the
// GhostFromCoarser comment below for the closed form).
template <int Q, class R>
__device__ __forceinline__ void compact_uloc(const R (&ul)[4][3], const R (&Sl)[4][Lat<Q>::NS], R (&uloc)[3]) {
  constexpr int D = Lat<Q>::D, NS = Lat<Q>::NS;
  uloc[0] = uloc[1] = uloc[2] = R(0);
  if (D == 3) {
    auto Dx = [&](int c) { return R(0.5) * (-Sl[0][c] + Sl[1][c] + Sl[2][c] - Sl[3][c]); };
    auto Dy = [&](int c) { return R(0.5) * (-Sl[0][c] + Sl[1][c] - Sl[2][c] + Sl[3][c]); };
    auto Dz = [&](int c) { return R(0.5) * (-Sl[0][c] - Sl[1][c] + Sl[2][c] + Sl[3][c]); };
    constexpr int XX = 0, YY = 1, ZZ = 2, XY = 3, YZ = 4, XZ = NS - 1;
    const R h3 = Dz(XY) + Dx(YZ) + Dy(XZ);
    const R sd[3] = {R(0.5) * Dx(XX) + Dy(XY) - R(0.5) * Dx(YY) + Dz(XZ) - R(0.5) * Dx(ZZ),
                     Dx(XY) - R(0.5) * Dy(XX) + R(0.5) * Dy(YY) + Dz(YZ) - R(0.5) * Dy(ZZ),
                     Dx(XZ) - R(0.5) * Dz(XX) + Dy(YZ) - R(0.5) * Dz(YY) + R(0.5) * Dz(ZZ)};
    const R so[3] = {Dy(XX) + Dz(XX) + h3 - R(2) * Dx(YZ), Dx(YY) + Dz(YY) + h3 - R(2) * Dy(XZ),
                     Dx(ZZ) + Dy(ZZ) + h3 - R(2) * Dz(XY)};
#pragma unroll
    for (int b = 0; b < 3; ++b)
      uloc[b] = R(0.625) * ul[0][b] + R(0.125) * (ul[1][b] + ul[2][b] + ul[3][b]) - R(0.1875) * sd[b] -
                R(0.0625) * so[b];
  } else {
    auto Dx = [&](int c) { return R(0.5) * (-Sl[0][c] + Sl[1][c] - Sl[2][c] + Sl[3][c]); };
    auto Dy = [&](int c) { return R(0.5) * (-Sl[0][c] - Sl[1][c] + Sl[2][c] + Sl[3][c]); };
    const R axx = R(0.5) * Dx(0), axy = Dy(0), ayy = Dy(2) - R(0.5) * Dx(1);
    const R bxx = Dx(2) - R(0.5) * Dy(0), byy = R(0.5) * Dy(1), bxy = Dx(1);
    uloc[0] = R(0.5) * ul[0][0] + R(0.25) * (ul[1][0] + ul[2][0]) - R(0.1875) * (axx + ayy) + R(0.0625) * axy;
    uloc[1] = R(0.5) * ul[0][1] + R(0.25) * (ul[1][1] + ul[2][1]) - R(0.1875) * (bxx + byy) + R(0.0625) * bxy;
  }
}

// ----------------------------------------------------------------- GhostFromCoarser
// Interpolation steps 2-5 (Sec. 2.2) for one fine ghost from its four coarse
// sources.  The velocity is the compact quadratic interpolant evaluated at the
// ghost, written in the octant's local frame (signs s_a) in closed form:
// 3D (H, K, M, N at (0,0,0), (1,1,0), (1,0,1), (0,1,1); ghost at (1/4,1/4,1/4)),
//   u_a = 5/8 u_H + 1/8 (u_K + u_M + u_N) - 3/16 (q_xx + q_yy + q_zz)_a
//         - 1/16 (q_xy + q_yz + q_xz)_a,
// with the quadratic coefficients q from the strain-rate differences of
// Eqs. (compact_3D_s); 2D (H, E, N, NE on the unit square, ghost at (1/4,1/4)),
//   u_a = 1/2 u_H + 1/4 (u_E + u_N) - 3/16 (q_xx + q_yy)_a + 1/16 q_xy,a,
// the least-squares linear part over the square.  Density and f^neq are
// linear (weights 5/8,1/8,1/8,1/8 resp. 9/16,3/16,3/16,1/16), f^neq is
// rescaled by omega_c / (m omega_f) (m = dt_c / dt_f), and f = f^eq +
// (1 - omega_f) f^neq is stored as the ghost's post-collision state.  With
// diffusive scaling the velocity and density deviation are converted to the
// fine level's lattice units first, and f^neq's odd part (a flux of order
// tau dt^2 / dx) takes an extra factor 1/2 beside its even part's.
// Ghosts come in groups of 2^d consecutive siblings (the children of one
// coarse parent, octant b = k mod 2^d), and their 4 x 2^d source records are
// 13 distinct ones in 3D (the parent and its 12 edge neighbours), 9 in 2D.  A
// group's lanes stage those records in shared memory with whole-record vector
// loads (one cache line per record), then each lane reads its four sources
// from there.
template <int D>
struct GfcGroup {
  static constexpr int G = 1 << D;           // lanes (siblings) per group
  static constexpr int NSLOT = D == 3 ? 13 : 9;
  // slot of source s (0: parent, 1-3 as in gsrc) for the sibling in octant b
  __device__ static int slot(int s, int b) {
    if (D == 3) return s == 0 ? 0 : s == 1 ? 1 + (b & 3) : s == 2 ? 5 + ((b & 1) | ((b >> 1) & 2)) : 9 + ((b >> 1) & 3);
    return s == 0 ? 0 : s == 1 ? 1 + (b & 1) : s == 2 ? 3 + ((b >> 1) & 1) : 5 + (b & 3);
  }
  // the (source, sibling) pair whose gsrc entry names slot t
  __host__ __device__ static constexpr int src_of(int t) { return t == 0 ? 0 : D == 3 ? 1 + (t - 1) / 4 : (t < 3 ? 1 : t < 5 ? 2 : 3); }
  __host__ __device__ static constexpr int lane_of(int t) {
    return D == 3 ? (t == 0 ? 0 : t < 5 ? t - 1 : t < 9 ? ((t - 5) & 1) | (((t - 5) & 2) << 1) : (t - 9) << 1)
                  : (t == 0 ? 0 : t < 3 ? t - 1 : t < 5 ? (t - 3) << 1 : t - 5);
  }
};

// Interpolation steps 2-5 for ghost k (octant oct) from its group's staged
// records (sg_base: NSLOT padded records), written into a.dst.
template <int Q, class S>
__device__ __forceinline__ void gfc_ghost(const GfcArgs& a, const typename Sto<S>::R* sg_base, int oct, int64_t k) {
  using R = typename Sto<S>::R;
  using LT = Lat<Q>;
  using RL = RecLayout<Q>;
  using GG = GfcGroup<LT::D>;
  constexpr int D = LT::D, NS = LT::NS;
  constexpr int PSTR = RL::STRIDE + 4;
  const R* rec[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) rec[s] = sg_base + GG::slot(s, oct) * PSTR;
  R sg[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) sg[c] = ((oct >> c) & 1) ? R(1) : R(-1);
  // local-frame velocity and strain rate of the sources (vector loads of the
  // record tail: rho, u, S)
  R ul[4][3], Sl[4][NS], rps[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    R h[RL::STRIDE - RL::RP];
#pragma unroll
    for (int f = RL::RP; f < RL::STRIDE; f += 4)
      if (f < RL::END) ld4(rec[s] + f, h + (f - RL::RP));
    rps[s] = h[0];
#pragma unroll
    for (int b = 0; b < D; ++b) ul[s][b] = sg[b] * h[RL::U - RL::RP + b];
#pragma unroll
    for (int b = 0; b < D; ++b)
#pragma unroll
      for (int c = b; c < D; ++c)
        Sl[s][sidx<D>(b, c)] = sg[b] * sg[c] * h[RL::SS - RL::RP + sidx<D>(b, c)];
  }
  R uloc[3];
  compact_uloc<Q, R>(ul, Sl, uloc);
  R u[3] = {R(0), R(0), R(0)};
  R usq = R(0);
  const R us = R(a.u_scale);  // to fine lattice units (1 in acoustic scaling)
#pragma unroll
  for (int b = 0; b < D; ++b) {
    u[b] = sg[b] * uloc[b] * us;
    usq += u[b] * u[b];
  }
  const R lw0 = D == 3 ? R(0.625) : R(0.5625);
  const R lw1 = D == 3 ? R(0.125) : R(0.1875);
  const R lw2 = D == 3 ? R(0.125) : R(0.1875);
  const R lw3 = D == 3 ? R(0.125) : R(0.0625);
  const R rp = R(a.r_scale) * (lw0 * rps[0] + lw1 * rps[1] + lw2 * rps[2] + lw3 * rps[3]) + R(a.r_shift);
  const R rho = R(a.rho_off) + rp;
  const R wf = R(a.omega_f);
  const R scale = (R(1) - wf) * R(a.omega_c) / (R(a.tratio) * wf);
  S* __restrict__ dst = static_cast<S*>(a.dst);
  const size_t N = (size_t)a.Ntot;
  const int64_t e = a.dest0 + k;
  // interpolated f^neq, then f^eq per pair of opposite velocities (shared even part)
  R fn[Q];
#pragma unroll
  for (int q0 = 0; q0 < Q; q0 += 4) {
    R f0[4], f1[4], f2[4], f3[4];
    ld4(rec[0] + RL::FN + q0, f0);
    ld4(rec[1] + RL::FN + q0, f1);
    ld4(rec[2] + RL::FN + q0, f2);
    ld4(rec[3] + RL::FN + q0, f3);
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (q0 + c < Q) fn[q0 + c] = lw0 * f0[c] + lw1 * f1[c] + lw2 * f2[c] + lw3 * f3[c];
  }
  const R base = rp - R(1.5) * rho * usq;
  dst[e] = Sto<S>::cv(R(LT::w(0)) * base + scale * fn[0]);
  // diffusive scaling: f^neq's odd part takes an extra factor (odd_ratio)
  const bool odd_rescale = a.odd_ratio != 1.0;
  const R ro = R(a.odd_ratio);
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    R cu = R(0);
#pragma unroll
    for (int b = 0; b < D; ++b) {
      if (LT::c(i, b) > 0) cu += u[b];
      if (LT::c(i, b) < 0) cu -= u[b];
    }
    const R w = R(LT::w(i));
    const R even = w * (base + R(4.5) * rho * cu * cu);
    const R odd = w * R(3) * rho * cu;
    R fa = fn[i], fb = fn[i + 1];
    if (odd_rescale) {
      const R fe = R(0.5) * (fa + fb), fo = R(0.5) * (fa - fb) * ro;
      fa = fe + fo;
      fb = fe - fo;
    }
    dst[(size_t)i * N + e] = Sto<S>::cv(even + odd + scale * fa);
    dst[(size_t)(i + 1) * N + e] = Sto<S>::cv(even - odd + scale * fb);
  }
}


#ifndef LBM_GFC_BLOCK
#define LBM_GFC_BLOCK 64
#endif
#if defined(LBM_GFC_MINB) && LBM_GFC_MINB > 0
#define LBM_GFC_BOUNDS __launch_bounds__(LBM_GFC_BLOCK, LBM_GFC_MINB)
#else
#define LBM_GFC_BOUNDS __launch_bounds__(LBM_GFC_BLOCK)
#endif
template <int Q, class S, bool TWO>
__global__ void LBM_GFC_BOUNDS k_fill_gfc(const GfcArgs a) {
  using R = typename Sto<S>::R;
  using LT = Lat<Q>;
  using RL = RecLayout<Q>;
  using GG = GfcGroup<LT::D>;
  constexpr int G = GG::G, NSLOT = GG::NSLOT;
  constexpr int PSTR = RL::STRIDE + 4;  // padded record: sibling lanes' reads fall in distinct banks
  constexpr int NGRP = LBM_GFC_BLOCK / G;
  __shared__ __align__(16) R stage[NGRP * NSLOT * PSTR];
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int oct = threadIdx.x & (G - 1);  // octant of the ghost
  const int grp = threadIdx.x / G;
  const bool active = k < a.ng;                   // ng is a multiple of G: whole groups
  const unsigned lane0 = (threadIdx.x & 31) & ~(unsigned)(G - 1);
  int32_t src[4] = {0, 0, 0, 0};
  if (active)
#pragma unroll
    for (int s = 0; s < 4; ++s) src[s] = a.gsrc[(size_t)s * a.ng + k];
  const R* __restrict__ mom = static_cast<const R*>(a.mom);
  const R* __restrict__ mom2 = static_cast<const R*>(a.mom2);
  R* sg_base = stage + grp * NSLOT * PSTR;
#pragma unroll
  for (int t = 0; t < NSLOT; ++t) {
    const int r = __shfl_sync(0xffffffffu, src[GG::src_of(t)], lane0 + GG::lane_of(t));
    if (active)
#pragma unroll
      for (int c = oct; c < RL::STRIDE / 4; c += G) {
        R v[4];
        ld4(mom + (size_t)r * RL::STRIDE + 4 * c, v);
        if (TWO) {
          // the records at t + 1/2: mean of those at t and t + 1
          R w[4];
          ld4(mom2 + (size_t)r * RL::STRIDE + 4 * c, w);
#pragma unroll
          for (int j = 0; j < 4; ++j) v[j] = R(0.5) * (v[j] + w[j]);
        }
        st4(sg_base + t * PSTR + 4 * c, v);
      }
  }
  __syncwarp();
  // outer-layer ghosts are staged with their group but, when skipped, not written
  if (!active || (a.skip_outer && (a.oct[k] & kGfcOuter))) return;
  gfc_ghost<Q, S>(a, sg_base, oct, k);
}

// ----------------------------------------------------------------- GhostFromFiner
// Coarse ghost from its 2^d children (Sec. 2.2 steps 1-5 with the children as
// sources; they surround the ghost symmetrically at +-1/4 coarse cell).
// Density and f^neq: the children's mean.  Velocity: the children's mean minus
// (1/32) lap u, with lap u_a = 2 d_c S_ac - d_a S_cc from the children's strain
// rates (differences across the children's cube).  f^neq is rescaled by
// m omega_f / omega_c (m = dt_c / dt_f); f = f^eq + (1 - omega_c) f^neq.  With
// diffusive scaling the mean velocity and density deviation are converted to
// the coarse level's lattice units, and f^neq's odd part takes an extra
// factor 2.
// One group of 2^d consecutive lanes per ghost: lane b loads child b (siblings
// are contiguous, so the group's loads are coalesced), and the sums over the
// children are shuffles inside the group.
#if defined(LBM_GFF_MINB) && LBM_GFF_MINB > 0
#define LBM_GFF_BOUNDS __launch_bounds__(256, LBM_GFF_MINB)
#else
#define LBM_GFF_BOUNDS __launch_bounds__(256)
#endif
template <int Q, class S, bool FORCE>
__global__ void LBM_GFF_BOUNDS k_fill_gff(const GffArgs a) {
  using R = typename Sto<S>::R;
  using LT = Lat<Q>;
  constexpr int D = LT::D, NS = LT::NS, NCH = 1 << D;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t k = t / NCH;
  const int b = (int)(t % NCH);
  const bool active = k < a.ng;
  const S* __restrict__ src = static_cast<const S*>(a.src_fine);
  const size_t N = (size_t)a.Ntot;
  const R wf = R(a.omega_f), rho_off = R(a.rho_off);
  R rp = R(0), u[3] = {R(0), R(0), R(0)}, fneq[Q], Sv[NS];
#pragma unroll
  for (int q = 0; q < Q; ++q) fneq[q] = R(0);
#pragma unroll
  for (int s = 0; s < NS; ++s) Sv[s] = R(0);
  if (active) {
    const int64_t e = (int64_t)a.child0[k] + b;
    R g[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) g[q] = Sto<S>::ld(src + (size_t)q * N + e);
    R F[3] = {R(0), R(0), R(0)};
    if (FORCE)
#pragma unroll
      for (int c = 0; c < D; ++c) F[c] = static_cast<const R*>(a.force)[(size_t)c * N + e];
    post_moments<Q, R, true, FORCE>(g, wf, rho_off, F, rp, u, fneq, Sv);
    if (a.odd_ratio != 1.0) {
      // diffusive scaling: f^neq's odd part takes an extra factor (the sum
      // over the children is linear, so each child's share is rescaled)
      const R ro = R(a.odd_ratio);
#pragma unroll
      for (int i = 1; i < Q; i += 2) {
        const R fe = R(0.5) * (fneq[i] + fneq[i + 1]), fo = R(0.5) * (fneq[i] - fneq[i + 1]) * ro;
        fneq[i] = fe + fo;
        fneq[i + 1] = fe - fo;
      }
    }
  }
  // The ghost's velocity, mean minus (1/32) lap u, is linear in the children's
  // values, and so is lap u_a = dfac sum_c (2 d_c S_ac - d_a S_cc) with d_c the
  // difference across the cube (+ for children with bit c set, - otherwise):
  // each lane forms its child's share and the group sums d + 1 values.
  // d_c S (coarse units): S_coarse = m S_fine (m = dt_c / dt_f); difference of
  // the two half-cubes over a distance of 1/2 coarse cell -> factor m 2^{2-D}.
  // The mean velocity goes to coarse units with u_scale (a power of two, so
  // inv_u is exact).
  const R inv = R(1) / R(NCH);
  const R inv_u = inv * R(a.u_scale);
  const R dfac = R(a.tratio) * R(D == 3 ? 0.5 : 1.0);
  R rpm = rp * inv, uP[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int aa = 0; aa < D; ++aa) {
    const R sa = ((b >> aa) & 1) ? R(1) : R(-1);
    R lap = R(0);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const R sc = ((b >> c) & 1) ? R(1) : R(-1);
      lap += dfac * (R(2) * sc * Sv[sidx<D>(aa, c)] - sa * Sv[sidx<D>(c, c)]);
    }
    uP[aa] = u[aa] * inv_u - lap * R(1.0 / 32.0);
  }
#pragma unroll
  for (int o = 1; o < NCH; o <<= 1) {
    rpm += __shfl_xor_sync(0xffffffffu, rpm, o);
#pragma unroll
    for (int c = 0; c < D; ++c) uP[c] += __shfl_xor_sync(0xffffffffu, uP[c], o);
  }
  // f^neq: reduce-scatter (recursive halving), lane b ends with the sums for
  // q = j 2^d + b; at half-width h a lane keeps the half of its columns on its
  // side of bit h and receives its partner's partial sums of that half
  constexpr int NR = (Q + NCH - 1) / NCH;
  R W[NR][NCH];
#pragma unroll
  for (int j = 0; j < NR; ++j)
#pragma unroll
    for (int c = 0; c < NCH; ++c) W[j][c] = j * NCH + c < Q ? fneq[j * NCH + c] : R(0);
#pragma unroll
  for (int h = NCH / 2; h >= 1; h >>= 1) {
    const bool hi = (b & h) != 0;
#pragma unroll
    for (int j = 0; j < NR; ++j)
#pragma unroll
      for (int c = 0; c < h; ++c) {
        const R send = hi ? W[j][c] : W[j][c + h];
        const R keep = hi ? W[j][c + h] : W[j][c];
        W[j][c] = keep + __shfl_xor_sync(0xffffffffu, send, h);
      }
  }
  if (!active) return;
  R usq = R(0);
#pragma unroll
  for (int aa = 0; aa < D; ++aa) usq += uP[aa] * uP[aa];
  const R wc = R(a.omega_c);
  rpm = R(a.r_scale) * rpm + R(a.r_shift);  // to coarse units (unchanged in acoustic scaling)
  const R rho = rho_off + rpm;
  const R scale = (R(1) - wc) * R(a.tratio) * wf / wc * inv;
  S* __restrict__ dst = static_cast<S*>(a.dst);
  const int64_t e = k < a.n_inner ? a.dest0 + k : a.dest_outer + (k - a.n_inner);
  // the group's lanes share the Q stores: lane b the directions j 2^d + b,
  // whose c_i it looks up at run time (a compile-time loop over all Q would
  // issue every direction's arithmetic in every lane)
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const int q = j * NCH + b;
    if (q < Q) {
      R cu = R(0);
#pragma unroll
      for (int aa = 0; aa < D; ++aa) cu += R(LatRt<Q>::c(q, aa)) * uP[aa];
      const R feq = LatRt<Q>::template w<R>(q) * (rpm + rho * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq));
      dst[(size_t)q * N + e] = Sto<S>::cv(feq + scale * W[j][0]);
    }
  }
}

// ----------------------------------------------------------------- set-up (compute type) / output (FP64)
template <int Q, class S>
__global__ void k_fill_rest(const FillArgs a) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.Ntot) return;
  S* p = static_cast<S*>(a.pdf);
#pragma unroll
  for (int q = 0; q < Q; ++q)
    p[(size_t)q * a.Ntot + e] = Sto<S>::cv(typename Sto<S>::R(Lat<Q>::w(q) * (a.rho0 - a.rho_off)));
}

// Initial state, Sec. 4.1: f = f^eq + (1 - omega) f^neq + df with
// f^neq_i = -(3 w_i rho / omega) (c_i c_i - I/3) : S.  HAS_S: a strain rate is
// given (a template flag, so that the loop over the directions has no branch
// on it and unrolls into compile-time lattice constants).
template <int Q, class S, bool HAS_S>
__global__ void k_init(const InitArgs a) {
  using R = typename Sto<S>::R;
  using LT = Lat<Q>;
  constexpr int D = LT::D, NS = LT::NS;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.cnt) return;
  const int64_t k = a.first + t;
  const int li = a.ulev[k];
  // equilibrium in the deviation form of the storage (g = f - w rho_off),
  // computed in the storage's compute type like the collision's equilibrium
  const R rho = R(a.rho[t]);
  const R rp = R(a.rho[t] - a.rho_off);
  R u[3] = {R(0), R(0), R(0)}, usq = R(0);
#pragma unroll
  for (int b = 0; b < D; ++b) {
    u[b] = R(a.u[t * D + b]);
    usq += u[b] * u[b];
  }
  R sv[NS], tr = R(0);
  if (HAS_S) {
#pragma unroll
    for (int j = 0; j < NS; ++j) sv[j] = R(a.S[t * NS + j]);
#pragma unroll
    for (int b = 0; b < D; ++b) tr += sv[sidx<D>(b, b)];
  }
  const double* df = a.df ? a.df + t * Q : nullptr;
  const R om = R(a.omega[li]);
  S* out = static_cast<S*>(a.temp) + k;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    R g = geq<Q, R>(q, rp, rho, u, usq);
    if (HAS_S) {
      R qs = R(0);
#pragma unroll
      for (int b = 0; b < D; ++b)
#pragma unroll
        for (int c = b; c < D; ++c) qs += R((b == c ? 1 : 2) * LT::c(q, b) * LT::c(q, c)) * sv[sidx<D>(b, c)];
      // post-collision non-equilibrium part (1 - omega) f^neq of the strain rate
      g += (R(1) - om) * (-(R(3.0 * LT::w(q)) * rho / om) * (qs - tr / R(3)));
    }
    if (df) g += R(df[q]);
    out[(size_t)q * a.n_user] = Sto<S>::cv(g);
  }
}

// caller-ordered initial pdfs -> element slots (coalesced writes in slot order)
template <int Q, class S>
__global__ void k_init_place(const PlaceArgs a) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.Ntot) return;
  const int32_t u = a.slot_user[e];
  if (u < 0) return;
  const S* src = static_cast<const S*>(a.temp) + u;
  S* dst = static_cast<S*>(a.dst) + e;
#pragma unroll
  for (int q = 0; q < Q; ++q) dst[(size_t)q * a.Ntot] = src[(size_t)q * a.n_user];
}

template <int Q, class S>
__global__ void k_out(const OutArgs a) {
  using LT = Lat<Q>;
  constexpr int D = LT::D, NS = LT::NS;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.cnt) return;
  const int64_t k = a.first + t;
  const int li = a.ulev[k];
  const S* cur = static_cast<const S*>(((a.parity >> li) & 1) ? a.B : a.A);
  const int64_t e = a.uslot[k];
  double g[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) g[q] = (double)Sto<S>::ld(cur + (size_t)q * a.Ntot + e);
  if (a.f) {
    double* o = a.f + t * Q;
#pragma unroll
    for (int q = 0; q < Q; ++q) o[q] = g[q] + LT::w(q) * a.rho_off;
  }
  if (!a.rho && !a.u && !a.S) return;
  double F[3] = {0, 0, 0};
  if (a.force) {
    // force is stored in the compute type
    if (sizeof(typename Sto<S>::R) == 8)
      for (int b = 0; b < D; ++b) F[b] = static_cast<const double*>(a.force)[(size_t)b * a.Ntot + e];
    else
      for (int b = 0; b < D; ++b) F[b] = static_cast<const float*>(a.force)[(size_t)b * a.Ntot + e];
  }
  double rp, u[3], fneq[Q], Sv[NS];
  post_moments<Q, double, true>(g, a.omega[li], a.rho_off, F, rp, u, fneq, Sv);
  if (a.rho) a.rho[t] = a.rho_off + rp;
  if (a.u)
#pragma unroll
    for (int b = 0; b < D; ++b) a.u[t * D + b] = u[b];
  if (a.S)
#pragma unroll
    for (int s = 0; s < NS; ++s) a.S[t * NS + s] = Sv[s];
}

template <int Q, class S>
__global__ void k_set_state(const SetStateArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.cnt) return;
  const int64_t k = a.first + t;
  const int li = a.ulev[k];
  S* cur = static_cast<S*>(((a.parity >> li) & 1) ? a.B : a.A);
  const int64_t e = a.uslot[k];
#pragma unroll
  for (int q = 0; q < Q; ++q)
    cur[(size_t)q * a.Ntot + e] =
        Sto<S>::cv(typename Sto<S>::R(a.f[t * Q + q] - Lat<Q>::w(q) * a.rho_off));
}

template <int Q, class S>
__global__ void k_gather_ghosts(const GatherGhostArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.cnt) return;
  const S* p = static_cast<const S*>(a.pdf);
#pragma unroll
  for (int q = 0; q < Q; ++q)
    a.stage[t * Q + q] = (double)Sto<S>::ld(p + (size_t)q * a.Ntot + a.first_global + t) + Lat<Q>::w(q) * a.rho_off;
}

// ----------------------------------------------------------------- FP64 reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int NV>
__device__ __forceinline__ void block_sum_store(double (&v)[NV], double* out) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    const double s = warp_sum(v[c]);
    if (lane == 0) sh[c][wid] = s;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      double s = lane < nw ? sh[c][lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) out[c] = s;
    }
  }
}

// Running sum of FP32 values kept as an unevaluated pair hi + lo (Knuth's
// two-sum: hi + x is split exactly into its rounded value and the rounding
// error, which lo collects): about twice the FP32 precision on the FP32
// pipe, converted to FP64 once at the end.
struct SumF2 {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// mass, momentum, obstacle force (momentum exchange, Sec. 2.3) and kinetic energy
// of one level; one partial row per block, fixed grid -> deterministic order.
// A thread sums its elements' moments (FP32 compute type: as two-float sums,
// which keeps the FP64 pipe, GB300's narrow one, out of the per-element work;
// FP64 storage: in FP64), then the block and grid sums are FP64.
template <int Q, class S>
__global__ void __launch_bounds__(256) k_reduce(const ReduceArgs a) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const S* p = static_cast<const S*>(a.pdf);
  const size_t N = (size_t)a.Ntot;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // each element's moments in the storage's compute type (the sums of its Q
  // stored values); the accumulation over elements in FP64
  // (the level volume and rho_off are applied once per thread below)
  using R = typename Sto<S>::R;
  constexpr bool F2 = sizeof(R) == 4;
  SumF2 sf[5];  // rp, rho u, kinetic energy (FP32 compute type)
  int64_t cnt = 0;
  for (int64_t e = a.begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.end; e += stride) {
    R g[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) g[q] = Sto<S>::ld(p + (size_t)q * N + e);
    R rp, j[3];
    raw_moments<Q, R>(g, rp, j);
    R F[3] = {R(0), R(0), R(0)};
    if (a.force)
      for (int b = 0; b < D; ++b) F[b] = static_cast<const R*>(a.force)[(size_t)b * N + e];
    const R rho = R(a.rho_off) + rp;
    R uu = R(0);
    R m[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int b = 0; b < D; ++b) {
      m[b] = j[b] - R(0.5) * F[b];  // rho u
      uu += m[b] * m[b];
    }
    const R ke = R(0.5) * uu / rho;
    if constexpr (F2) {
      sf[0].add(rp);
#pragma unroll
      for (int b = 0; b < D; ++b) sf[1 + b].add(m[b]);
      sf[4].add(ke);
    } else {
      acc[0] += (double)rp;
#pragma unroll
      for (int b = 0; b < D; ++b) acc[1 + b] += (double)m[b];
      acc[7] += (double)ke;
    }
    ++cnt;
  }
  if constexpr (F2) {
    acc[0] = sf[0].value();
#pragma unroll
    for (int b = 0; b < 3; ++b) acc[1 + b] = sf[1 + b].value();
    acc[7] = sf[4].value();
  }
  if (a.r_scale == 1.0)
    acc[0] = a.vol * (acc[0] + (double)cnt * a.rho_off);
  else  // density deviations in another level's units
    acc[0] = a.vol * ((double)cnt * a.rho0 + a.r_scale * (acc[0] + (double)cnt * (a.rho_off - a.rho0)));
#pragma unroll
  for (int b = 0; b < 3; ++b) acc[1 + b] *= a.vol_m;
  acc[7] *= a.vol_k;
  // momentum exchange (Sec. 2.3): the link carries c_ib (f*_ib(x) + f_i(x)) to
  // the body, f_i the bounce-back value of the next step (interpolated with
  // the wall distance q; q = 1/2 gives 2 c_ib f*_ib)
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < a.obs_n; l += stride) {
    const int i = a.obs_dir[l];
    const int ib = opp(i);
    const int64_t e = a.obs_elem[l];
    const double q = a.obs_q ? a.obs_q[l] : 0.5;
    const double go = (double)Sto<S>::ld(p + (size_t)ib * N + e);
    double gb;
    if (q < 0.5) {
      const int32_t a2 = a.obs_a ? a.obs_a[l] : -1;
      gb = a2 < 0 ? go : 2.0 * q * go + (1.0 - 2.0 * q) * (double)Sto<S>::ld(p + (size_t)ib * N + a2);
    } else {
      gb = go / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * (double)Sto<S>::ld(p + (size_t)i * N + e);
    }
    const double sum = go + gb + 2.0 * LT::w(ib) * a.rho_off;
#pragma unroll
    for (int b = 0; b < D; ++b) acc[4 + b] += a.fscale * LT::c(ib, b) * sum;
  }
  block_sum_store<8>(acc, a.partial + (size_t)blockIdx.x * 8);
}

// ----------------------------------------------------------------- launchers
inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Calls f with std::integral_constant<int, Q> for the run-time stencil Q
// (9, 19 or 27; the mesh builder rejects anything else).
template <class F>
inline void with_q(int Q, F&& f) {
  if (Q == 9) f(std::integral_constant<int, 9>{});
  else if (Q == 19) f(std::integral_constant<int, 19>{});
  else f(std::integral_constant<int, 27>{});
}

template <class S>
struct Launch {
  static void stream_collide_brick(int Q, bool force, bool boundary, const BrickArgs& a, cudaStream_t st) {
    if (a.nB <= 0) return;
    const unsigned g = blocks_for(a.nB, LBM_BR_BLOCK / 64);
    with_q(Q, [&](auto q) {
      constexpr int QQ = decltype(q)::value;
      const bool moms = a.so.mask != nullptr;
      if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        // BF16 interior bricks: two elements per thread, one brick per warp
        // (on levels without GFC sources; the others take the one-element
        // kernel with its record epilogue)
        if (!boundary && !moms) {
          const unsigned g2 = blocks_for(a.nB, LBM_BR_PAIR_BLOCK / 32);
          if (force) k_stream_collide_brick_pair<QQ, true><<<g2, LBM_BR_PAIR_BLOCK, 0, st>>>(a);
          else k_stream_collide_brick_pair<QQ, false><<<g2, LBM_BR_PAIR_BLOCK, 0, st>>>(a);
          return;
        }
      }
      auto go = [&](auto F, auto B, auto M) {
        k_stream_collide_brick<QQ, S, decltype(F)::value, decltype(B)::value, decltype(M)::value>
            <<<g, LBM_BR_BLOCK, 0, st>>>(a);
      };
      using T = std::true_type;
      using U = std::false_type;
      if (boundary) {
        if (force) moms ? go(T{}, T{}, T{}) : go(T{}, T{}, U{});
        else moms ? go(U{}, T{}, T{}) : go(U{}, T{}, U{});
      } else {
        if (force) moms ? go(T{}, U{}, T{}) : go(T{}, U{}, U{});
        else moms ? go(U{}, U{}, T{}) : go(U{}, U{}, U{});
      }
    });
  }
  static void stream_collide(int Q, bool force, const StreamCollideArgs& a, cudaStream_t st) {
    const int64_t n = a.end - a.begin;
    if (n <= 0) return;
    constexpr int EPT = LBM_SC_EPT;
    const unsigned g = blocks_for(n, LBM_SC_BLOCK * EPT);
    with_q(Q, [&](auto q) {
      constexpr int QQ = decltype(q)::value;
      const bool moms = a.so.mask != nullptr;
      if (force) {
        if (moms) k_stream_collide<QQ, S, true, EPT, true><<<g, LBM_SC_BLOCK, 0, st>>>(a);
        else k_stream_collide<QQ, S, true, EPT, false><<<g, LBM_SC_BLOCK, 0, st>>>(a);
      } else {
        if (moms) k_stream_collide<QQ, S, false, EPT, true><<<g, LBM_SC_BLOCK, 0, st>>>(a);
        else k_stream_collide<QQ, S, false, EPT, false><<<g, LBM_SC_BLOCK, 0, st>>>(a);
      }
    });
  }
  static void outlet(int Q, const OutletArgs& a, cudaStream_t st) {
    const int64_t n = a.end - a.begin;
    if (n <= 0) return;
    with_q(Q, [&](auto q) { k_outlet<decltype(q)::value, S><<<blocks_for(n, 128), 128, 0, st>>>(a); });
  }
  static void source_moments(int Q, const MomentsArgs& a, cudaStream_t st) {
    if (a.nsrc <= 0) return;
    with_q(Q, [&](auto q) {
      constexpr int QQ = decltype(q)::value;
      const unsigned g = blocks_for(a.nsrc, LBM_MOM_BLOCK);
      if (a.force) k_source_moments<QQ, S, true><<<g, LBM_MOM_BLOCK, 0, st>>>(a);
      else k_source_moments<QQ, S, false><<<g, LBM_MOM_BLOCK, 0, st>>>(a);
    });
  }
  static void fill_gfc(int Q, const GfcArgs& a, cudaStream_t st) {
    if (a.ng <= 0) return;
    with_q(Q, [&](auto q) {
      constexpr int QQ = decltype(q)::value;
      const unsigned g = blocks_for(a.ng, LBM_GFC_BLOCK);
      if (a.mom2) k_fill_gfc<QQ, S, true><<<g, LBM_GFC_BLOCK, 0, st>>>(a);
      else k_fill_gfc<QQ, S, false><<<g, LBM_GFC_BLOCK, 0, st>>>(a);
    });
  }
  static void fill_gff(int Q, const GffArgs& a, cudaStream_t st) {
    if (a.ng <= 0) return;
    with_q(Q, [&](auto q) {
      constexpr int QQ = decltype(q)::value;
      const unsigned g = blocks_for(a.ng * (1 << Lat<QQ>::D), 256);
      if (a.force) k_fill_gff<QQ, S, true><<<g, 256, 0, st>>>(a);
      else k_fill_gff<QQ, S, false><<<g, 256, 0, st>>>(a);
    });
  }
  static void fill_rest(int Q, const FillArgs& a, cudaStream_t st) {
    with_q(Q, [&](auto q) { k_fill_rest<decltype(q)::value, S><<<blocks_for(a.Ntot, 256), 256, 0, st>>>(a); });
  }
  static void init(int Q, const InitArgs& a, cudaStream_t st) {
    if (a.cnt <= 0) return;
    with_q(Q, [&](auto q) {
      if (a.S) k_init<decltype(q)::value, S, true><<<blocks_for(a.cnt, 128), 128, 0, st>>>(a);
      else k_init<decltype(q)::value, S, false><<<blocks_for(a.cnt, 128), 128, 0, st>>>(a);
    });
  }
  static void init_place(int Q, const PlaceArgs& a, cudaStream_t st) {
    with_q(Q, [&](auto q) { k_init_place<decltype(q)::value, S><<<blocks_for(a.Ntot, 256), 256, 0, st>>>(a); });
  }
  static void out(int Q, const OutArgs& a, cudaStream_t st) {
    if (a.cnt <= 0) return;
    with_q(Q, [&](auto q) { k_out<decltype(q)::value, S><<<blocks_for(a.cnt, 128), 128, 0, st>>>(a); });
  }
  static void set_state(int Q, const SetStateArgs& a, cudaStream_t st) {
    if (a.cnt <= 0) return;
    with_q(Q, [&](auto q) { k_set_state<decltype(q)::value, S><<<blocks_for(a.cnt, 128), 128, 0, st>>>(a); });
  }
  static void gather_ghosts(int Q, const GatherGhostArgs& a, cudaStream_t st) {
    if (a.cnt <= 0) return;
    with_q(Q, [&](auto q) { k_gather_ghosts<decltype(q)::value, S><<<blocks_for(a.cnt, 128), 128, 0, st>>>(a); });
  }
  static void reduce(int Q, const ReduceArgs& a, cudaStream_t st) {
    with_q(Q, [&](auto q) { k_reduce<decltype(q)::value, S><<<a.nblocks, 256, 0, st>>>(a); });
  }
};

template <class S>
const Ops* make_ops() {
  static const Ops ops = {&Launch<S>::stream_collide, &Launch<S>::stream_collide_brick,
                          &Launch<S>::outlet,         &Launch<S>::source_moments,
                          &Launch<S>::fill_gfc,       &Launch<S>::fill_gff,   &Launch<S>::fill_rest,
                          &Launch<S>::init,           &Launch<S>::init_place, &Launch<S>::out,
                          &Launch<S>::set_state,
                          &Launch<S>::gather_ghosts,
                          &Launch<S>::reduce,         sizeof(S),              sizeof(typename Sto<S>::R),
                          // every storage type streams its boundary bricks through the
                          // brick tables (BF16: 2.85 against 5.50 ms per sphere step
                          // through the neighbour list, measured)
                          true};
  return &ops;
}

}  // namespace dev
}  // namespace lbm
