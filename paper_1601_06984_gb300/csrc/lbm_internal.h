// Internal structures of liblbm: host mesh tables, the device workspace layout
// and the kernel launch interface.  Not part of the public ABI (include/lbm.h).
#pragma once

#include <cuda_runtime_api.h>

#include <climits>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "lbm.h"

namespace lbm {

// Neighbour (pull) index encoding, one uint32 per element and direction i >= 1:
//   bit31=0 bit30=0 : pull f_i from global element index (bits 0..29) of the same level
//   bit31=1 bit30=0 : half-way bounce-back, read the element's own f_opp(i)
//   bit31=1 bit30=1 : velocity bounce-back (inlet): own f_opp(i) + 6 w_i rho0 (c_i . u_in)
//   bit31=0 bit30=1 : precomputed incoming value (outlet), index into the boundary values
constexpr uint32_t NB_BOUNCE = 0x80000000u;
constexpr uint32_t NB_FLAG30 = 0x40000000u;
constexpr uint32_t NB_INDEX = 0x3FFFFFFFu;
constexpr int kPad = 32;  // every level segment is padded to a multiple of this
static_assert(kPad % 32 == 0, "source masks take 32-slot blocks inside one level");
constexpr int32_t kBrickMissing = INT32_MIN;  // brick row entry: neighbour brick not complete
constexpr uint8_t kGfcOuter = 0x80;  // GhostFromCoarser octant byte: ghost of the outer layer

enum { K_FLUID = 0, K_GFC = 1, K_GFF = 2, K_PAD = 3 };

// Discrete velocities in the order documented in lbm.h (D2Q9, D3Q19, and
// D3Q27 = D3Q19 followed by the corners in opposite pairs) and the standard
// weights by |c|^2 (Sec. 2.1): D2Q9 4/9, 1/9, 1/36; D3Q19 1/3, 1/18, 1/36;
// D3Q27 8/27, 2/27, 1/54, 1/216.  The one host copy of the lattice.
constexpr int kQmax = 27;
inline void host_lattice(int Q, int c[kQmax][3], double w[kQmax]) {
  static const int c27[27][3] = {{0, 0, 0},   {1, 0, 0},    {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},  {0, 0, 1},
                                 {0, 0, -1},  {1, 1, 0},    {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},  {1, 0, 1},
                                 {-1, 0, -1}, {1, 0, -1},   {-1, 0, 1}, {0, 1, 1},   {0, -1, -1}, {0, 1, -1},
                                 {0, -1, 1},  {1, 1, 1},    {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1}, {1, -1, 1},
                                 {-1, 1, -1}, {-1, 1, 1},   {1, -1, -1}};
  // D2Q9 order: rest, +x, -x, +y, -y, (+x+y), (-x-y), (+x-y), (-x+y)
  static const int c9[9][3] = {{0, 0, 0}, {1, 0, 0},  {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                               {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
  for (int i = 0; i < kQmax; ++i) {
    for (int a = 0; a < 3; ++a) c[i][a] = i < Q ? (Q == 9 ? c9[i][a] : c27[i][a]) : 0;
    const int n2 = c[i][0] * c[i][0] + c[i][1] * c[i][1] + c[i][2] * c[i][2];
    if (i >= Q) w[i] = 0.0;
    else if (Q == 9) w[i] = n2 == 0 ? 4.0 / 9.0 : (n2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
    else if (Q == 19) w[i] = n2 == 0 ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    else w[i] = n2 == 0 ? 8.0 / 27.0 : (n2 == 1 ? 2.0 / 27.0 : (n2 == 2 ? 1.0 / 54.0 : 1.0 / 216.0));
  }
}
enum { OUT_NORMAL = 0, OUT_EXTRAP = 1, OUT_BOUZIDI = 2 };

// Time scaling of a level interface (Sec. 2.2).  Acoustic scaling (LINEAR and
// TWO_LAYER modes): dt_c / dt_f = 2, two fine substeps, and the relaxation
// follows Eq. (fneq_scale), 1/w_f - 1/2 = 2 (1/w_c - 1/2).  Diffusive scaling
// (dt proportional to dx^2): dt_c / dt_f = 4, four fine substeps, the lattice
// viscosity and so omega the same on every level; a level's lattice velocity
// is (dt/dx) times the physical one, so u_c = 2 u_f for the same flow, the
// density deviation (a pressure) goes with u^2, and the strain rate with dt.
inline int time_ratio(int mode) { return mode == LBM_TIME_DIFFUSIVE ? 4 : 2; }
inline double finer_omega(double omega_c, int mode) {
  return mode == LBM_TIME_DIFFUSIVE ? omega_c : 1.0 / (0.5 + 2.0 * (1.0 / omega_c - 0.5));
}
// f^neq's odd part in c (a flux of order tau dt^2 / dx) changes between levels
// by (dt_f / dt_c) / (dx_f / dx_c) more than its even part (the stress, of
// order tau dt) that Eq. (fneq_scale) rescales: the extra factor, 1 with
// acoustic scaling, 1/2 coarse to fine and 2 fine to coarse with diffusive
// scaling
inline double odd_fneq_ratio(int mode, bool to_coarse) {
  return mode != LBM_TIME_DIFFUSIVE ? 1.0 : to_coarse ? 2.0 : 0.5;
}
// the same flow's lattice velocity on level index li over that on the coarsest level
inline double level_velocity_ratio(int li, int mode) { return mode == LBM_TIME_DIFFUSIVE ? std::ldexp(1.0, -li) : 1.0; }

struct HostLevel {
  int L = 0;
  double omega = 1.0;
  int64_t nC = 0, nF = 0, nG1 = 0, nG2 = 0;  // GFC, fluid, GFF inner layer, GFF outer layer
  int64_t oC = 0, oF = 0, oG1 = 0, oG2 = 0;  // padded segment offsets (local)
  int64_t N = 0;                             // padded local size
  int64_t base = 0;                          // global index of local element 0
  // ghosts (host copies for lbm_get_ghosts): coords and layer per ghost, GFC then GFF
  std::vector<int32_t> ghost_xyz;  // [nC + nG1 + nG2][3]
  std::vector<int8_t> ghost_layer;
  // GhostFromFiner of this level: global index of the first child on level L+1
  std::vector<int32_t> gff_child0;  // [nG1 + nG2]
  // GhostFromCoarser of this level: 4 positions in the source list of level L-1, octant bits
  std::vector<int32_t> gfc_src;  // [4][nC]
  std::vector<uint8_t> gfc_oct;  // [nC], bit a < 3 set: ghost on the + side of its parent along a;
                                 // kGfcOuter: outer layer (no fluid or subdivided neighbour)
  // sources (global indices on this level) feeding the GFC of level L+1
  std::vector<int32_t> src_elem;
  // sources that are GhostFromFiner ghosts (their records follow the ghost
  // fill): element and record index, the inner layer first
  std::vector<int32_t> gsrc_elem, gsrc_rec;
  int64_t n_gsrc_inner = 0;
  // outlet links processed before this level's stream-collide: global range in the outlet list
  int64_t out_begin = 0, out_end = 0;
  // obstacle links of this level: global range in the obstacle list
  int64_t obs_begin = 0, obs_end = 0;
  // bricks: the first 64 nB fluid elements are interior bricks, the next
  // 64 nBb boundary bricks; their rows in brick_nb from brick_first
  int64_t nB = 0, nBb = 0, brick_first = 0;
};

struct HostMesh {
  int d = 2, Q = 9, nS = 3;
  int Lmin = 0, Lmax = 0;
  int64_t n_user = 0;
  int64_t Ntot = 0;
  std::vector<HostLevel> lv;
  std::vector<uint32_t> nbr;    // [Q-1][Ntot]
  std::vector<int32_t> uslot;   // [n_user] global element index
  std::vector<int32_t> slot_user;  // [Ntot] caller index of each slot, -1 for ghosts and padding
  std::vector<uint8_t> ulev;    // [n_user] level index (L - Lmin)
  std::vector<uint8_t> kind;    // [Ntot] element kind (K_*)
  // boundary-value links (all levels, grouped by level): outlet links and, with
  // interpolated bounce-back, obstacle links; a, b: extrapolation sources or the
  // second node x + c_i of an obstacle link (-1: none); q: wall distance
  std::vector<int32_t> out_elem, out_a, out_b;
  std::vector<int8_t> out_dir, out_kind;
  std::vector<double> out_q;
  // obstacle links (all levels, grouped by level): element, direction i with
  // x - c_i solid, second node x + c_i (-1: none), wall distance q, and the
  // link's boundary-value index (-1 with half-way bounce-back)
  std::vector<int32_t> obs_elem, obs_a, obs_side;
  std::vector<int8_t> obs_dir;
  std::vector<double> obs_q;
  // inlet links: velocity profile factor per link (nbr low bits index it)
  std::vector<double> inlet_s;
  // interior bricks (64 elements each, z-curve order inside): per brick the
  // first element of the brick at offset slot t = (sx+1) + 3 (sy+1) + 9 (sz+1),
  // relative to the brick's own first element (slot 13, the brick itself, is
  // 0); per link i >= 1 and local position l the entry (t << 6) | l' locating
  // the pull source f*_i(x - c_i) at first + brick_nb[t] + l'
  std::vector<int32_t> brick_nb;    // [sum nB][27]
  std::vector<uint16_t> brick_tab;  // [Q-1][64]
  // GhostFromCoarser sources, per 32 slots (level segments are 32-aligned, so
  // a block lies in one level): bit j set if slot 32 blk + j is a source of
  // its level, and the record index of the block's first source
  std::vector<uint32_t> src_mask;  // [Ntot / 32]
  std::vector<int32_t> src_first;  // [Ntot / 32]
};

// Build the mesh tables; returns LBM_OK or LBM_ERR_MESH / LBM_ERR_ARG with msg.
lbm_status build_host_mesh(const int64_t* tree_ids, const int8_t* levels, int64_t n,
                           const lbm_params& p, HostMesh* out, std::string* msg);

// Sec. 3.1 utility (host only).
lbm_status sfc_partition(const int64_t* tree_ids, int64_t n, int d, int nparts, int64_t* order,
                         int64_t* weights, int64_t* cumulative, int32_t* part, std::string* msg);

// ----------------------------------------------------------------- kernels
// Launch arguments are plain data; pointers are device pointers into the
// workspace.  "src"/"dst" are pdf arrays [Q][Ntot] of the storage type.
// GFC source records written by a stream-collide (interpolation step 1 of
// Sec. 2.2 fused into the kernel that produces the source state): for every
// processed element marked in mask, the record of its new state goes to
// rec_out.  mask null: no records.
struct SourceOut {
  const uint32_t* mask;  // [Ntot / 32] source bits per 32 slots
  const int32_t* first;  // [Ntot / 32] record index of each block's first source
  void* rec_out;         // [nsrc][mom_stride(Q)] records of the new state
};
struct StreamCollideArgs {
  const void* src;
  void* dst;
  const uint32_t* nbr;
  const void* force;  // [d][Ntot] compute type, or null
  const void* side;   // boundary values, compute type, or null
  const double* inlet_s;  // inlet profile factor per inlet link
  int64_t Ntot, begin, end;  // linear range; element = lin + (lin >= hole_at ? hole_len : 0)
  int64_t hole_at, hole_len;  // interior bricks skipped by this kernel (0 length: none)
  double omega, rho_off;
  double inlet[kQmax];  // 6 w_i rho0 (c_i . u_in)
  SourceOut so;
};

// Stream-collide of the interior bricks of one level: nB bricks of 64
// elements from global index begin; neighbour bricks and link table as in
// HostMesh::brick_nb / brick_tab.
struct BrickArgs {
  const void* src;
  void* dst;
  const void* force;    // [d][Ntot] compute type, or null
  const int32_t* nb;    // [nB][27] rows (offsets from the brick's first element, or kBrickMissing)
  const uint16_t* tab;  // [Q-1][64]
  int64_t Ntot, begin, nB;
  double omega, rho_off;
  // boundary bricks: links through a missing neighbour brick use the element's
  // neighbour-list code (pull, bounce-back, inlet, boundary value)
  const uint32_t* nbr;
  const void* side;
  const double* inlet_s;
  double inlet[kQmax];
  SourceOut so;
};

struct OutletArgs {
  const void* src;
  void* side;
  const int32_t *elem, *a, *b;
  const int8_t *dir, *kind;
  const void* force;
  int64_t Ntot, begin, end;
  double omega, rho_off, rho0;
  int zero_gradient;  // extrapolate with f(x - n) instead of 2 f(x - n) - f(x - 2n)
  const double* q;    // wall distance of interpolated bounce-back links
};

// GFC source moments: one record of mom_stride(Q) values per source (compute
// type): f^neq[Q] padded to a multiple of 4, rho - rho_off, u[d], S[nS], zero
// padding.
constexpr int mom_stride(int Q) { return Q == 27 ? 40 : 32; }
struct MomentsArgs {
  const void* src;
  const void* force;
  const int32_t* elem;
  void* mom;         // [nsrc][mom_stride(Q)]
  const void* prev;  // if set: mom = (prev + moments now) / 2 (mean of two time levels)
  const int32_t* rec;  // record index of elem[k] (null: k)
  int64_t Ntot, nsrc;
  double omega, rho_off;
};

struct GfcArgs {
  const void* mom;       // [nsrc][mom_stride(Q)] source records
  const void* mom2;      // if set: the records are the means of mom and mom2 (t + 1/2)
  int64_t nsrc;
  const int32_t* gsrc;   // [4][ng]
  const uint8_t* oct;    // [ng]
  int64_t ng, dest0;     // global index of the first GFC
  void* dst;
  int64_t Ntot;
  double omega_c, omega_f, rho_off;
  int skip_outer;        // leave the outer-layer ghosts (oct & kGfcOuter) unwritten
  // unit conversion coarse -> fine: dt_c / dt_f, u_f = u_scale u_c and the
  // density deviation rho'_f = r_scale rho'_c + r_shift (relative to rho_off);
  // odd_ratio: the extra factor of f^neq's odd part (odd_fneq_ratio)
  double tratio, u_scale, r_scale, r_shift, odd_ratio;
};

struct GffArgs {
  const void* src_fine;  // pdfs holding the children
  const void* force;
  const int32_t* child0; // [ng], inner layer first
  int64_t ng, n_inner;   // ghosts k < n_inner go to dest0 + k, the rest to dest_outer + (k - n_inner)
  int64_t dest0, dest_outer;
  void* dst;             // pdfs holding the coarse ghosts
  int64_t Ntot;
  double omega_c, omega_f, rho_off;
  // unit conversion fine -> coarse: dt_c / dt_f, u_c = u_scale u_f and the
  // density deviation rho'_c = r_scale rho'_f + r_shift (relative to rho_off);
  // odd_ratio: the extra factor of f^neq's odd part (odd_fneq_ratio)
  double tratio, u_scale, r_scale, r_shift, odd_ratio;
};

struct FillArgs {  // rest equilibrium everywhere
  void* pdf;
  int64_t Ntot;
  double rho0, rho_off;
};

struct InitArgs {  // initial pdfs of a chunk of caller-order elements, written caller-ordered
  void* temp;        // [Q][n_user] storage type (the pdf buffer that is not current)
  const uint8_t* ulev;
  const double *rho, *u, *S, *df;  // staged chunk: rho[cnt], u[cnt][d], S[cnt][nS] or null, df[cnt][Q] or null
  int64_t first, cnt, n_user;
  double omega[16];
  double rho_off;
};

struct PlaceArgs {  // caller-ordered pdfs -> element slots of the current buffer
  const void* temp;  // [Q][n_user]
  void* dst;         // [Q][Ntot]
  const int32_t* slot_user;  // [Ntot] caller index of each slot, -1 for ghosts and padding
  int64_t n_user, Ntot;
};

struct SetStateArgs {  // FP64 [cnt][Q] in user order -> current pdfs
  void* A;
  void* B;
  const int32_t* uslot;
  const uint8_t* ulev;
  uint32_t parity;
  const double* f;
  int64_t first, cnt, Ntot;
  double rho_off;
};

struct OutArgs {  // moments / state to FP64 staging in user order
  const void* A;
  const void* B;
  const void* force;
  const int32_t* uslot;
  const uint8_t* ulev;
  uint32_t parity;
  double *rho, *u, *S, *f;  // staged chunk outputs (any may be null)
  int64_t first, cnt, Ntot;
  double omega[16];
  double rho_off;
};

struct ForceArgs {  // scatter user force to [d][Ntot]
  void* force;
  const int32_t* uslot;
  const double* stage;  // [cnt][d]
  int64_t first, cnt, Ntot;
  int dim;
};

struct GatherGhostArgs {  // ghost pdfs -> FP64 [cnt][Q]
  const void* pdf;
  int64_t first_global, cnt, Ntot;
  double* stage;
  double rho_off;
};

struct ReduceArgs {
  const void* pdf;       // current state of the level
  const void* force;
  int64_t Ntot, begin, end;  // fluid range of the level
  double omega, rho_off, vol;
  double* partial;       // [nblocks][8]
  int nblocks;
  // obstacle links of the level
  const int32_t* obs_elem;
  const int8_t* obs_dir;
  const int32_t* obs_a;   // second node of the interpolated bounce-back (-1: none)
  const double* obs_q;    // wall distance (1/2: half-way bounce-back)
  int64_t obs_n;
  double fscale;
  // mass vol (cnt rho0 + r_scale sum (rho - rho0)) (r_scale 1: vol sum rho),
  // momentum vol_m sum rho u, kinetic energy vol_k sum rho |u|^2 / 2
  double vol_m, vol_k, r_scale, rho0;
};

struct FinalArgs {
  const double* partial;
  int64_t n;  // partial rows
  double* out;
};

struct Ops {
  void (*stream_collide)(int Q, bool force, const StreamCollideArgs&, cudaStream_t);
  void (*stream_collide_brick)(int Q, bool force, bool boundary, const BrickArgs&, cudaStream_t);
  void (*outlet)(int Q, const OutletArgs&, cudaStream_t);
  void (*source_moments)(int Q, const MomentsArgs&, cudaStream_t);
  void (*fill_gfc)(int Q, const GfcArgs&, cudaStream_t);
  void (*fill_gff)(int Q, const GffArgs&, cudaStream_t);
  void (*fill_rest)(int Q, const FillArgs&, cudaStream_t);
  void (*init)(int Q, const InitArgs&, cudaStream_t);
  void (*init_place)(int Q, const PlaceArgs&, cudaStream_t);
  void (*out)(int Q, const OutArgs&, cudaStream_t);
  void (*set_state)(int Q, const SetStateArgs&, cudaStream_t);
  void (*gather_ghosts)(int Q, const GatherGhostArgs&, cudaStream_t);
  void (*reduce)(int Q, const ReduceArgs&, cudaStream_t);
  size_t storage_bytes;  // bytes per stored pdf
  size_t compute_bytes;  // bytes of the compute type
  bool boundary_bricks;  // stream boundary bricks with the brick kernel (else with the neighbour list)
};

// ----------------------------------------------------------------- adjoint kernels
// lam* are adjoint pdf buffers [Q][Ntot] in the compute type; lam_force is
// [d][Ntot] FP64; partial holds one running row of parameter derivatives per
// block (cols 0..15 d/d omega of each level, 16..18 d/d u_in): block b of
// every launch adds its sums to row b, so the totals are deterministic.
constexpr int kAdjBlocks = 1024;  // fixed grid of the adjoint kernels (deterministic partials)
#define LBM_BRICKS_PER_BLOCK 4       // bricks of 64 elements per 256-thread block of the brick kernels
constexpr int kAccCols = 32;

struct AdjCommon {
  const void* fsrc;   // forward state the op read (full [Q][Ntot] snapshot, storage type)
  const void* force;  // [d][Ntot] compute type or null (treated as zero force)
  void* lam_a;        // adjoint buffer the op's outputs live in (consumed, zeroed)
  void* lam_b;        // adjoint buffer of the op's inputs (accumulated)
  double* lam_force;  // [d][Ntot] FP64 accumulated (null: not wanted)
  double* partial;    // [kAdjBlocks][kAccCols] running sums
  int64_t Ntot;
  double rho_off, rho0;
  int la, lb;         // levels whose omega the launch's first / second sums belong to (lb < 0: none)
};

struct AdjSCArgs {
  AdjCommon c;
  const uint32_t* nbr;
  const void* side_fwd;  // outlet values the forward used (compute type)
  void* lam_side;        // adjoint of the outlet values (written)
  int64_t begin, end;    // neighbour-list kernel: linear range; element = lin + (lin >= hole_at ? hole_len : 0)
  int64_t hole_at, hole_len;
  double omega;
  double inlet[kQmax];   // 6 w_i rho0 (c_i . u_in) of the forward
  const double* inlet_s;  // inlet profile factor per inlet link
  // interior-brick kernel: nB bricks of 64 elements from begin, their rows
  // [nB][27] and the link table [Q-1][64] (as BrickArgs)
  const int32_t* brick_nb;
  const uint16_t* brick_tab;
  int64_t nB;
};

struct AdjOutletArgs {
  AdjCommon c;
  const int32_t *elem, *a, *b;
  const int8_t *dir, *kind;
  const void* lam_side;
  int64_t begin, end;
  // outlet links: 0 normal links, 1 extrapolation term of source a, 2 of source b;
  // interpolated bounce-back links: 3 term f*_i(x), 4 term f*_ib(x), 5 term f*_ib(x + c_i)
  int which;
  double omega;
  int zero_gradient;
  const double* q;
};

struct AdjMomArgs {  // reverse of the source moments
  AdjCommon c;       // lam_b: adjoint of the coarse state
  const int32_t* elem;
  void* lam_rec;       // [nsrc][mom_stride(Q)] adjoint of the records (consumed, zeroed)
  void* lam_rec_prev;  // averaging mode: receives half of lam_rec (else null)
  int64_t nsrc;
  double omega;
};

struct AdjGfcArgs {  // reverse of the GhostFromCoarser fill, per ghost
  AdjCommon c;       // lam_a: adjoint of the fine state holding the ghosts
  const void* rec;   // forward source records [nsrc][mom_stride(Q)]
  const int32_t* gsrc;
  const uint8_t* oct;
  void* contrib;     // [ng][4][mom_stride(Q)] per-ghost adjoint of each source record
  int64_t ng, dest0;
  double omega_c, omega_f;
};

struct AdjGatherArgs {  // deterministic sum of the per-ghost contributions per source
  const void* contrib;
  const int32_t* off;   // [nsrc+1]
  const int32_t* item;  // ghost*4 + source slot
  void* lam_rec;        // [nsrc][stride] accumulated
  int64_t nsrc;
  int stride;           // mom_stride(Q): 32 or 40
};

struct AdjGffArgs {
  AdjCommon c;       // fsrc: fine state (children); lam_a: coarse adjoint; lam_b: fine adjoint
  const int32_t* child0;
  int64_t ng, n_inner, dest0, dest_outer;
  double omega_c, omega_f;
};

struct AdjSeedArgs {
  AdjCommon c;  // lam_b receives the seed
  int objective;  // 0 kinetic energy; 1..3 obstacle force x, y, z
  int64_t begin, end;  // fluid range (kinetic energy)
  double vol;
  const int32_t* obs_elem;
  const int8_t* obs_dir;
  const int32_t* obs_a;
  const double* obs_q;
  int64_t obs_n;
  double fscale;
  int which;  // force objective: 0 the link's own slot, 1 its second node, 2 the opposite slot
};

struct AccumArgs {
  const double* partial;  // [rows][kAccCols]
  int rows;
  double* acc;            // [kAccCols] column sums (assigned)
};

struct AdjOps {
  void (*seed)(int Q, const AdjSeedArgs&, cudaStream_t);
  void (*sc)(int Q, const AdjSCArgs&, cudaStream_t);
  void (*sc_brick)(int Q, const AdjSCArgs&, cudaStream_t);  // grid ceil(nB / 4) blocks
  void (*outlet)(int Q, const AdjOutletArgs&, cudaStream_t);
  void (*moments)(int Q, const AdjMomArgs&, cudaStream_t);
  void (*gfc)(int Q, const AdjGfcArgs&, cudaStream_t);
  void (*gff)(int Q, const AdjGffArgs&, cudaStream_t);
  size_t lam_bytes;  // bytes per adjoint value (compute type)
};
const AdjOps* adj_ops_fp64();
const AdjOps* adj_ops_fp32dev();
const AdjOps* adj_ops_bf16dev();
void launch_adj_gather(bool fp64, const AdjGatherArgs&, cudaStream_t);
void launch_accum(const AccumArgs&, cudaStream_t);
// Copies bytes [off, off + len) of each of `rows` rows of pitch `pitch` from
// src to dst (same layout); elem is the element size the offsets are multiples of.
void launch_copy_rows(const void* src, void* dst, size_t pitch, size_t off, size_t len, int rows, size_t elem,
                      cudaStream_t);
void launch_gather_lam_user(bool fp64, const void* lamA, const void* lamB, uint32_t parity, const int32_t* uslot,
                            const uint8_t* ulev, double* stage, int64_t first, int64_t cnt, int64_t Ntot, int Q,
                            cudaStream_t);
void launch_gather_force_user(const double* lam_force, const int32_t* uslot, double* stage, int64_t first,
                              int64_t cnt, int64_t Ntot, int d, cudaStream_t);

const Ops* ops_fp64();
const Ops* ops_fp32dev();
const Ops* ops_bf16dev();
void launch_scatter_force(bool fp64, const ForceArgs&, cudaStream_t);
void launch_final_reduce(const FinalArgs&, cudaStream_t);
constexpr int kReduceBlocks = 512;  // blocks per reduce launch (fixed: deterministic order)

// What a reduction over a bound context needs, without the scratch pointers
// (used by the entry point that keeps its scratch in a static device array).
struct ReducePlan {
  const Ops* ops = nullptr;
  int Q = 0;
  cudaStream_t stream = nullptr;
  const void* workspace = nullptr;
  std::vector<ReduceArgs> levels;  // partial == nullptr; filled in by the caller
};
lbm_status reduce_plan(lbm_ctx* ctx, ReducePlan* plan);
lbm_status set_error(lbm_ctx* ctx, lbm_status s, const std::string& msg);
void count_launches(lbm_ctx* ctx, int64_t n);

}  // namespace lbm
