// Walk kernels of the swap-neighbourhood QAP search (sm_103a).
//
// One CTA runs one search walk at a time and loops over walks (persistent
// form).  Per walk everything lives on chip:
//   shared memory   F (int8 when every difference of two F entries and of
//                   two D entries fits a byte, else int16) and, for an
//                   asymmetric flow, F^T; P = D[p][p] (int8) and, for
//                   asymmetric distances, P^T (kNoTransposed plans keep no
//                   transposed copies); the tabu marks (int32 per pair);
//                   the O(1)-update vectors; two recomputed delta rows;
//                   g[k] = sum_j F[k][j]P[k][j] + F[j][k]P[j][k] (double-
//                   buffered), or the products M of which g is the
//                   diagonal (kProductM plans, where P stays the walk's
//                   starting P0 and labels sigma track the locations); p
//                   and the best permutation.
//   registers       the delta of every pair the thread owns: a segment of
//                   at most MAXPT consecutive pairs (u, v) of one row u
//                   (large-n plans keep them in a per-CTA workspace).
//
// One tabu iteration, move (r, s) already chosen, has two barriers:
//   phase X  (reads the pre-move P, called Q below)  one task per index k:
//            k outside {r, s}: the Eq. 2 deltas of pairs {r, k} and {s, k}
//            after the move, from dot products of F / F^T rows with Q / Q^T
//            rows (dp4a for int8 F, dp2a for int16 F) or read from M, plus
//            O(1) corrections; the update vectors of k; g'[k].
//            k in {r, s}: g'[k].
//   -- barrier --
//   phase Y  owners update their deltas: pairs disjoint from {r, s} by
//            delta += (a_u-a_v)(b_u-b_v) + (c_u-c_v)(e_u-e_v) with
//              a_x = F[r][x]-F[s][x], b_x = P'[s][x]-P'[r][x],
//              c_x = F[x][r]-F[x][s], e_x = P'[x][s]-P'[x][r]
//            (one dp4a of byte vectors on the int8 path); pairs touching r
//            or s from the recomputed rows; pair (r, s) negated; each
//            updated delta enters the scan of the next iteration (tabu /
//            aspiration filter, lowest (rank, r, s)).  Rows and columns r, s
//            of P (and P^T) are then exchanged and p[r], p[s] swapped; with
//            kProductM p[r], p[s] and sigma[r], sigma[s] are swapped instead
//            and every thread brings its share of M up to date.
//   -- barrier --  (inside the CTA arg-min: warp REDUX, then one round
//                   through shared memory)
// Dot products over all j count the j = x and j = k terms; removing them and
// adding the two fixed terms of Eq. 2 leaves one product,
//   (F[x][x]-F[x][k]-F[k][x]+F[k][k]) (P'[x][x]-P'[x][k]-P'[k][x]+P'[k][k]).
// The dot with a post-move row is the dot with the pre-move row plus a
// correction for the two exchanged columns.
#pragma once
#include <climits>
#include <cstdint>
#include <type_traits>

#include "qap_philox.cuh"

namespace qapk {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kNoMove = 0xffffffffu;
constexpr int kDescentCap = 1 << 20;      // 2opt moves when no cap is given

// One instance as the kernels see it.
struct InstArgs {
  int n, ldF, ldP;    // ldF: elements per F row; ldP: elements per P row
  int symF, symD;
  int group;          // lanes per phase-X task (1, 2, 4 or 8)
  int diff16;         // differences of two F entries fit int16, of two D entries int8
  const void* F;      // n x ldF (int8, int16 or int64), row-major, zero padded
  const void* Ft;     // transpose of F (== F when symF)
  const void* D;      // n x n, row-major (int8, or int64 with int64 flows)
};

// Search parameters and per-walk outputs (rows indexed by output row).
struct SearchArgs {
  uint32_t walk_base; // walk id of a walk = walk_base + its index in its instance
  uint64_t seed;
  int descend, max_descent, iters;
  int tmin, tmax, period, aspiration;
  int tenure_per_n;   // tmin, tmax, period in hundredths of the instance's n
  int crit;           // tabu criterion: 0 pair (r, s), 1 unit-location, 2 unit
  int lambda;         // frequency penalty on non-improving moves (0 = off)
  size_t rws_off;     // offset of the criterion/penalty tables in a CTA's workspace
  size_t p_off;       // offset of P (then P^T) in a CTA's workspace (kGlobalP plans)
  int p_stride;       // elements per best_p row
  int32_t* best_p;
  int64_t* best_cost;
  int64_t* final_cost;
  int32_t* best_iter;
  int32_t* iters_done;
  int32_t* status;
  int32_t* descent_moves;
  uint64_t* hash;
  uint64_t* descent_hash;
  int32_t* freq;      // p_stride x p_stride per row, or null
};

// Walks of one instance.
struct WalkArgs {
  InstArgs inst;
  SearchArgs s;
  unsigned char* ws;      // large-n plans: per-CTA workspace (deltas, tabu stamps)
  size_t ws_stride;       // bytes per CTA
  int walks;              // walks processed by this launch
  int walk_offset;        // index of this launch's first walk among the instance's walks
  const int32_t* starts;  // (walk_offset + walks) x n, or null
};

// Walks of many instances in one launch: work item i (in longest-first
// order) is walk item_walk[i] of instance item_inst[i]; its output row is
// row_base[inst] + walk.  CTAs take items from a device counter.
struct BatchArgs {
  const InstArgs* insts;
  const int32_t* item_inst;
  const int32_t* item_walk;
  const int32_t* row_base;
  int items;
  int* counter;           // zeroed before the launch
  SearchArgs s;
  unsigned char* ws;      // large-n plans: per-CTA workspace (deltas, tabu stamps)
  size_t ws_stride;       // bytes per CTA
};

// Where a plan keeps its state.  Register plans hold each thread's deltas in
// registers and the tabu stamps in shared memory.  Large-n plans (bit
// kGlobalDelta) keep both in a per-CTA workspace in global memory, read and
// written coalesced (slot i of thread t at i * NT + t), so that F and P of n
// up to 256 fit in shared memory; with bit kGlobalFlow they also read F and
// F^T from global memory (L1-cached), leaving shared memory to P and P^T.
constexpr int kGlobalDelta = 1;
constexpr int kGlobalFlow = 2;
// Plans with bit kProductM (int8 or int16 flows) keep the n x n products
//   M[x][k] = sum_j F[x][j] P[k][j] + F[j][x] P[j][k]
// in shared memory, their columns indexed by unit (see compute_m), and
// update them after each move (see phase_m_update), so that phase X reads
// the dot products it needs instead of computing them.
constexpr int kProductM = 4;
// Plans with bit kGlobalP (int64 elements only) keep P and P^T in the CTA's
// workspace (at SearchArgs::p_off) instead of shared memory; they read F and
// F^T from global memory too.
constexpr int kGlobalP = 8;
// Products plans with bit kNoTransposed keep no transposed copies of F and P
// in shared memory (room for M on large asymmetric instances): the few
// transposed reads, at the start of a walk and in phase X, read columns.
constexpr int kNoTransposed = 16;

// row stride of M in int32 words: whole 16-byte groups, an odd number of
// them (rows read side by side by consecutive threads spread over banks)
__host__ __device__ inline int ld_m(int n) { return 4 * (((n + 3) / 4) | 1); }
// int32 words per index of the products form's update vectors: int8 flows
// pack (b, e, a, c) into one word; int16 flows keep (a, c) and (b, e) as
// int32 pairs (differences of int16 values need 17 bits)
__host__ __device__ constexpr int m_words(int fbytes) { return fbytes == 1 ? 1 : 2; }

// ---------------------------------------------------------------------------
// shared-memory layout (host and device agree through this function)
// ---------------------------------------------------------------------------
struct SmemLayout {
  int offF, offFt, offP, offPt, offTabu, offVec, offR, offG0, offG1, offPerm, offBest, offRedD,
      offRedK, offSum, offM;
  int bytes;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

// fbytes: bytes per F element (1, 2, or 8 for the int64 element path, whose
// P and update vectors are int64 too)
__host__ __device__ inline SmemLayout smem_layout(int n, int ldF, int fbytes, int ldP, int symF,
                                                  int symD, int dbytes, int slots,
                                                  int store = 0) {
  SmemLayout L;
  int o = 0;
  const bool fg = store & kGlobalFlow;
  const bool pg = store & kGlobalP;
  const int pbytes = fbytes == 8 ? 8 : 1;   // P element
  const int vbytes = fbytes == 8 ? 32 : 16; // update vector (a, b, c, e) of one index
  if (store & kGlobalDelta) slots = 0;
  L.offF = o;    o = fg ? o : align16(o + n * ldF * fbytes);
  const bool nt = store & kNoTransposed;
  L.offFt = o;   o = (symF || fg || nt) ? o : align16(o + n * ldF * fbytes);
  L.offP = o;    o = pg ? o : align16(o + n * ldP * pbytes);
  L.offPt = o;   o = (symD || pg || nt) ? o : align16(o + n * ldP * pbytes);
  L.offTabu = o; o = align16(o + slots * 4);
  L.offVec = o;  o = align16(o + n * vbytes);
  L.offR = o;    o = align16(o + 2 * n * dbytes);
  L.offG0 = o;   o = align16(o + n * dbytes);
  L.offG1 = o;   o = align16(o + n * dbytes);
  L.offPerm = o; o = align16(o + n * 4);
  L.offBest = o; o = align16(o + n * 4);
  L.offRedD = o; o = align16(o + 32 * 8);
  L.offRedK = o; o = align16(o + 32 * 4);
  L.offSum = o;  o = align16(o + 32 * 8);
  // M, the update words by index and by label, and sigma (see compute_m)
  L.offM = o;
  o = (store & kProductM) ? align16(o + ((n + 2 * m_words(fbytes)) * ld_m(n) + n) * 4) : o;
  L.bytes = o;
  return L;
}

template <typename DT> struct DeltaMax;
template <> struct DeltaMax<int32_t> { static constexpr int32_t v = INT_MAX; };
template <> struct DeltaMax<int64_t> { static constexpr int64_t v = LLONG_MAX; };
template <typename DT> struct DeltaMin;
template <> struct DeltaMin<int32_t> { static constexpr int32_t v = INT_MIN; };
template <> struct DeltaMin<int64_t> { static constexpr int64_t v = LLONG_MIN; };

// Element types: F is stored as FE, P (and D) as Elem<FE>::P; differences,
// products and dot-product sums of elements are Elem<FE>::S.  The narrow
// paths (int8 or int16 flows, int8 distances) keep S in 32 bits: the host
// admits an instance to them only when every such sum fits, 2 n max|F|
// max|D| < 2^31.  The wide path stores F and D as int64 and computes in
// int64; the host admits it while the cost bound stays below 2^62, so that
// no sum, delta or cost difference leaves int64.
template <typename FE> struct Elem;
template <> struct Elem<int8_t> { using P = int8_t; using S = int; };
template <> struct Elem<int16_t> { using P = int8_t; using S = int; };
template <> struct Elem<int64_t> { using P = int64_t; using S = int64_t; };

// ---------------------------------------------------------------------------
// row chunks: F rows as int8 (16 per chunk, dp4a) or int16 (8, dp2a)
// ---------------------------------------------------------------------------
template <typename FE> struct Chunk;

template <> struct Chunk<int8_t> {
  static constexpr int W = 16;
  using FV = int4;
  using QV = int4;
  __device__ __forceinline__ static int dot(const FV f, const QV q, int acc) {
    acc = __dp4a(f.x, q.x, acc);
    acc = __dp4a(f.y, q.y, acc);
    acc = __dp4a(f.z, q.z, acc);
    return __dp4a(f.w, q.w, acc);
  }
};

template <> struct Chunk<int16_t> {
  static constexpr int W = 8;
  using FV = int4;
  using QV = int2;
  __device__ __forceinline__ static int dot(const FV f, const QV q, int acc) {
    acc = __dp2a_lo(f.x, q.x, acc);
    acc = __dp2a_hi(f.y, q.x, acc);
    acc = __dp2a_lo(f.z, q.y, acc);
    return __dp2a_hi(f.w, q.y, acc);
  }
};

// int64 flows and distances: two elements per 16-byte chunk
template <> struct Chunk<int64_t> {
  static constexpr int W = 2;
  using FV = longlong2;
  using QV = longlong2;
  __device__ __forceinline__ static int64_t dot(const FV f, const QV q, int64_t acc) {
    return acc + f.x * q.x + f.y * q.y;
  }
};

// ---------------------------------------------------------------------------
// O(1)-update vectors (a, b, c, e) of one index: four bytes and one int32
// in 8 bytes when the flows are int8 (see VecOps<int8_t>), else four int32
// ---------------------------------------------------------------------------
template <typename FE> struct VecOps;

// The O(1) update of a pair (u, v) disjoint from the move,
//   d + (a_u - a_v)(b_u - b_v) + (c_u - c_v)(e_u - e_v),
// from the per-index vectors (a, b, c, e) that phase X writes.
//
// int8 flows: the host admits them only when every difference of two F
// entries and of two D entries fits a byte, so a, b, c, e are bytes.
// Expanding the products, the update is w_u + w_v - (a_u b_v + c_u e_v +
// b_u a_v + e_u c_v) with w_x = a_x b_x + c_x e_x: one dp4a of the bytes
// (a_u, c_u, b_u, e_u) with (b_v, e_v, a_v, c_v).  Index x stores the
// second form and w_x; the owner of row u permutes its own bytes once.
template <> struct VecOps<int8_t> {
  using V = int2;                  // (bytes b, e, a, c; w)
  struct U { int A, w; };          // (bytes a, c, b, e; w) of the row index u
  __device__ __forceinline__ static V pack(int a, int b, int c, int e) {
    const uint32_t x = ((uint32_t)b & 0xffu) | (((uint32_t)e & 0xffu) << 8) |
                       (((uint32_t)a & 0xffu) << 16) | ((uint32_t)c << 24);
    return make_int2((int)x, a * b + c * e);
  }
  __device__ __forceinline__ static U prep(const V u) {
    return U{(int)__byte_perm((uint32_t)u.x, 0u, 0x1032u), u.y};
  }
  template <typename DT>
  __device__ __forceinline__ static DT update(const U& u, const V v, DT d) {
    // wrap-around sums: only the final value is bounded
    return (DT)((uint32_t)d + (uint32_t)u.w + (uint32_t)v.y - (uint32_t)__dp4a(u.A, v.x, 0));
  }
  __device__ __forceinline__ static void put(void* vec, int, int k, V v) {
    reinterpret_cast<V*>(vec)[k] = v;
  }
  __device__ __forceinline__ static V get(const void* vec, int, int k) {
    return reinterpret_cast<const V*>(vec)[k];
  }
};

// int8 flows, the word alone: index x stores only the bytes (b, e, a, c),
// and each reader recomputes w_x with one dp4a against (a, c, 0, 0).  Each
// slot then loads 4 bytes instead of 8 (shorter per-thread strides, fewer
// bank conflicts) at two more instructions.  Measured faster on the
// 6-slot products plan only (n = 50 asymmetric, 256 walks: 10.05 -> 9.82 ms
// per step); 0.2-2 % slower on the other int8 plans measured.
struct VecOpsWord : VecOps<int8_t> {
  __device__ __forceinline__ static void put(void* vec, int, int k, V v) {
    reinterpret_cast<int*>(vec)[k] = v.x;
  }
  __device__ __forceinline__ static V get(const void* vec, int, int k) {
    const int x = reinterpret_cast<const int*>(vec)[k];
    return make_int2(x, __dp4a(x, (int)__byte_perm((uint32_t)x, 0u, 0x4432u), 0));
  }
};

template <> struct VecOps<int16_t> {
  using V = int4;                  // (a, b, c, e)
  using U = int4;
  __device__ __forceinline__ static V pack(int a, int b, int c, int e) {
    return make_int4(a, b, c, e);
  }
  __device__ __forceinline__ static U prep(const V u) { return u; }
  template <typename DT>
  __device__ __forceinline__ static DT update(const U& u, const V v, DT d) {
    return d + (DT)((u.x - v.x) * (u.y - v.y) + (u.z - v.z) * (u.w - v.w));
  }
  __device__ __forceinline__ static void put(void* vec, int, int k, V v) {
    reinterpret_cast<V*>(vec)[k] = v;
  }
  __device__ __forceinline__ static V get(const void* vec, int, int k) {
    return reinterpret_cast<const V*>(vec)[k];
  }
};

// int64 elements: (a, b, c, e) as four int64 in 32 bytes
struct alignas(16) Vec64 {
  long long a, b, c, e;
};

template <> struct VecOps<int64_t> {
  using V = Vec64;
  using U = Vec64;
  __device__ __forceinline__ static V pack(int64_t a, int64_t b, int64_t c, int64_t e) {
    return V{a, b, c, e};
  }
  __device__ __forceinline__ static U prep(const V u) { return u; }
  template <typename DT>
  __device__ __forceinline__ static DT update(const U& u, const V v, DT d) {
    return d + (DT)((u.a - v.a) * (u.b - v.b) + (u.c - v.c) * (u.e - v.e));
  }
  __device__ __forceinline__ static void put(void* vec, int, int k, V v) {
    reinterpret_cast<V*>(vec)[k] = v;
  }
  __device__ __forceinline__ static V get(const void* vec, int, int k) {
    return reinterpret_cast<const V*>(vec)[k];
  }
};

// ---------------------------------------------------------------------------
// arg-min of (delta, key) across a warp, then across the CTA
// ---------------------------------------------------------------------------
__device__ __forceinline__ void warp_argmin(int32_t& d, uint32_t& k) {
  const int32_t m = __reduce_min_sync(kFull, d);
  k = __reduce_min_sync(kFull, d == m ? k : kNoMove);
  d = m;
}

__device__ __forceinline__ void warp_argmin(int64_t& d, uint32_t& k) {
  const int32_t hi = (int32_t)(d >> 32);
  const uint32_t lo = (uint32_t)d;
  const int32_t mh = __reduce_min_sync(kFull, hi);
  const uint32_t ml = __reduce_min_sync(kFull, hi == mh ? lo : 0xffffffffu);
  k = __reduce_min_sync(kFull, (hi == mh && lo == ml) ? k : kNoMove);
  d = (int64_t)(((uint64_t)(uint32_t)mh << 32) | ml);
}

template <typename DT, int NT>
__device__ __forceinline__ void block_argmin(DT& d, uint32_t& k, DT* redD, uint32_t* redK) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_argmin(d, k);
  if (lane == 0) {
    redD[warp] = d;
    redK[warp] = k;
  }
  __syncthreads();
  d = lane < NW ? redD[lane] : DeltaMax<DT>::v;
  k = lane < NW ? redK[lane] : kNoMove;
  warp_argmin(d, k);
}

template <int NT>
__device__ __forceinline__ int64_t block_sum(int64_t v, int64_t* red) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  v = lane < NW ? red[lane] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  __syncthreads();
  return v;
}

__device__ __forceinline__ uint64_t fnv_step(uint64_t h, uint32_t r, uint32_t s) {
  return (h ^ (uint64_t)((r << 16) | s)) * 1099511628211ull;
}


// ---------------------------------------------------------------------------
// per-walk state views
// ---------------------------------------------------------------------------
template <typename DT, typename FE>
struct WalkSmem {
  FE* F;
  FE* Ft;
  typename Elem<FE>::P* P;
  typename Elem<FE>::P* Pt;
  int32_t* tabu;
  void* vec;  // VecOps<FE>::V per index
  DT* R;
  DT* g0;
  DT* g1;
  int32_t* perm;
  int32_t* best;
  DT* redD;
  uint32_t* redK;
  int64_t* sum;
  int32_t* M;  // kProductM plans: M (n x ld_m(n)), update words by index and by label, sigma (n)
};

// Eq. 2 (with the diagonal term) for the pair {x, k}, by one thread, from the
// current P.  The column terms read the transposed copies so every access is
// along a row (NOTR: no copies, the columns themselves, stride ld).  Used for
// the initial deltas of a walk.
template <typename DT, typename FE, bool NOTR>
__device__ __forceinline__ DT delta_serial(const WalkSmem<DT, FE>& S, int n, int ldF, int ldP,
                                           bool sym, int x, int k) {
  using PE = typename Elem<FE>::P;
  using SC = typename Elem<FE>::S;
  const FE* Fx = S.F + x * ldF;
  const FE* Fk = S.F + k * ldF;
  const PE* Px = S.P + x * ldP;
  const PE* Pk = S.P + k * ldP;
  const FE* Ftx = NOTR ? S.F + x : S.Ft + x * ldF;
  const FE* Ftk = NOTR ? S.F + k : S.Ft + k * ldF;
  const PE* Ptx = NOTR ? S.P + x : S.Pt + x * ldP;
  const PE* Ptk = NOTR ? S.P + k : S.Pt + k * ldP;
  const int fs = NOTR ? ldF : 1, ps = NOTR ? ldP : 1;
  DT acc = 0;
  for (int j = 0; j < n; ++j) {
    if (j == x || j == k) continue;
    const SC t1 = ((SC)Fx[j] - (SC)Fk[j]) * ((SC)Pk[j] - (SC)Px[j]);
    if (sym) {
      acc += (DT)(2 * t1);
    } else {
      const SC t2 = ((SC)Ftx[j * fs] - (SC)Ftk[j * fs]) * ((SC)Ptk[j * ps] - (SC)Ptx[j * ps]);
      acc += (DT)t1 + (DT)t2;
    }
  }
  const SC fixed = ((SC)Fx[k] - (SC)Fk[x]) * ((SC)Pk[x] - (SC)Px[k]);
  const SC diag = ((SC)Fx[x] - (SC)Fk[k]) * ((SC)Pk[k] - (SC)Px[x]);
  return acc + (DT)fixed + (DT)diag;
}

// g[k] for every k from the current P (one task per k, lanes over chunks).
template <typename DT, typename FE, int NT>
__device__ __forceinline__ void compute_g(const WalkSmem<DT, FE>& S, DT* g, int n, int ldF,
                                          int ldP, bool sym, int G) {
  using C = Chunk<FE>;
  const int lg = threadIdx.x & (G - 1);
  const int grp = threadIdx.x / G;
  const int NG = NT / G;
  const int nc = (n + C::W - 1) / C::W;
  for (int base = 0; base < n; base += NG) {  // whole CTA per round (runs once per walk)
    const int k = min(base + grp, n - 1);
    const auto* Fk = reinterpret_cast<const typename C::FV*>(S.F + k * ldF);
    const auto* Pk = reinterpret_cast<const typename C::QV*>(S.P + k * ldP);
    const auto* Ftk = reinterpret_cast<const typename C::FV*>(S.Ft + k * ldF);
    const auto* Ptk = reinterpret_cast<const typename C::QV*>(S.Pt + k * ldP);
    typename Elem<FE>::S acc = 0;
    for (int c = lg; c < nc; c += G) {
      acc = C::dot(Fk[c], Pk[c], acc);
      if (!sym) acc = C::dot(Ftk[c], Ptk[c], acc);
    }
    for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (lg == 0 && base + grp < n) g[k] = sym ? (DT)2 * (DT)acc : (DT)acc;
  }
}

// Phase X of move (r, s): see the file header.  One task per index k, G
// lanes per task splitting the row chunks; the k-row chunks serve both rows
// {r, k} and {s, k}.  Tasks k = r and k = s compute g'[r] and g'[s].  After a
// reduce-scatter over the group, lane 0 finishes row {r, k} and lane 1 row
// {s, k} (lane 0 both when G = 1).  Reads Q = P before the move and gc = g of
// the pre-move state; writes vec, R (without the -g'[x] term) and gn.
template <typename DT, typename FE, int NT>
__device__ __forceinline__ void phase_x(const WalkSmem<DT, FE>& S, const DT* gc, DT* gn, int n,
                                        int ldF, int ldP, bool sym, int G, int r, int s) {
  using C = Chunk<FE>;
  using FV = typename C::FV;
  using QV = typename C::QV;
  using VO = VecOps<FE>;
  using PE = typename Elem<FE>::P;
  using SC = typename Elem<FE>::S;
  const int lg = threadIdx.x & (G - 1);
  const int grp = threadIdx.x / G;
  const int NG = NT / G;
  const int nc = (n + C::W - 1) / C::W;
  const FE* F = S.F;
  const PE* Q = S.P;
  const FE* Ft = S.Ft;
  const PE* Qt = S.Pt;
  const FV* Fr = reinterpret_cast<const FV*>(F + r * ldF);
  const FV* Fs = reinterpret_cast<const FV*>(F + s * ldF);
  const FV* Ftr = reinterpret_cast<const FV*>(Ft + r * ldF);
  const FV* Fts = reinterpret_cast<const FV*>(Ft + s * ldF);
  const QV* Qr = reinterpret_cast<const QV*>(Q + r * ldP);
  const QV* Qs = reinterpret_cast<const QV*>(Q + s * ldP);
  const QV* Qtr = reinterpret_cast<const QV*>(Qt + r * ldP);
  const QV* Qts = reinterpret_cast<const QV*>(Qt + s * ldP);
  // 2x2 blocks of F and Q at {r, s}
  const SC fRR = F[r * ldF + r], fRS = F[r * ldF + s];
  const SC fSR = F[s * ldF + r], fSS = F[s * ldF + s];
  const SC qRR = Q[r * ldP + r], qRS = Q[r * ldP + s];
  const SC qSR = Q[s * ldP + r], qSS = Q[s * ldP + s];
  // Up to 512 threads the bound is the same for every lane of a warp (its
  // first group), so whole warps run each round and the reductions use
  // full-warp shuffles; lanes past n work on row n - 1 and store nothing.
  // At 1024 threads (measured faster) each group runs its own rounds and
  // shuffles within the group.
  constexpr bool kWarpRounds = NT < 1024;
  const int nb = kWarpRounds ? n - (threadIdx.x & ~31) / G : n - grp;
  const unsigned smask =
      kWarpRounds ? kFull : ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
  for (int base = 0; base < nb; base += NG) {
    const int k0 = base + grp;
    const int k = min(k0, n - 1);
    const bool gt = (k == r) | (k == s);
    // k-task: Ar = F[r].Q[k] + F^T[r].Q^T[k]   Br = F[k].Q[s] + F^T[k].Q^T[s]
    //         As = F[s].Q[k] + F^T[s].Q^T[k]   Bs = F[k].Q[r] + F^T[k].Q^T[r]
    // g-task k = r: Ar with the row s in place of k; k = s: As with row r
    const int kq = gt ? (k == r ? s : r) : k;
    const FV* Fk = reinterpret_cast<const FV*>(F + kq * ldF);
    const FV* Ftk = reinterpret_cast<const FV*>(Ft + kq * ldF);
    const QV* Qk = reinterpret_cast<const QV*>(Q + kq * ldP);
    const QV* Qtk = reinterpret_cast<const QV*>(Qt + kq * ldP);
    SC Ar = 0, Br = 0, As = 0, Bs = 0;
    if (sym) {
      for (int c = lg; c < nc; c += G) {
        const FV fk = Fk[c];
        const QV qk = Qk[c];
        Ar = C::dot(Fr[c], qk, Ar);
        As = C::dot(Fs[c], qk, As);
        Br = C::dot(fk, Qs[c], Br);
        Bs = C::dot(fk, Qr[c], Bs);
      }
    } else {
      for (int c = lg; c < nc; c += G) {
        const FV fk = Fk[c], ftk = Ftk[c];
        const QV qk = Qk[c], qtk = Qtk[c];
        Ar = C::dot(Fr[c], qk, Ar);
        Ar = C::dot(Ftr[c], qtk, Ar);
        As = C::dot(Fs[c], qk, As);
        As = C::dot(Fts[c], qtk, As);
        Br = C::dot(fk, Qs[c], Br);
        Br = C::dot(ftk, Qts[c], Br);
        Bs = C::dot(fk, Qr[c], Bs);
        Bs = C::dot(ftk, Qtr[c], Bs);
      }
    }
    // reduce-scatter: even lanes gather (Ar, Br), odd lanes (As, Bs)
    const bool odd = lg & 1;
    SC A = odd ? As : Ar, B = odd ? Bs : Br;
    if (G > 1) {
      A += __shfl_xor_sync(smask, odd ? Ar : As, 1);
      B += __shfl_xor_sync(smask, odd ? Br : Bs, 1);
      for (int o = 2; o < G; o <<= 1) {
        A += __shfl_xor_sync(smask, A, o);
        B += __shfl_xor_sync(smask, B, o);
      }
    }
    if (k0 >= n || lg > 1) continue;
    if (gt) {
      // g'[x] = A + (F[x][r]-F[x][s])(Q[xb][s]-Q[xb][r])
      //           + (F[r][x]-F[s][x])(Q[s][xb]-Q[r][xb])
      const bool xs = (k == s);
      if (lg != ((G > 1 && xs) ? 1 : 0)) continue;  // the lane holding Ar or As
      const SC A0 = (G > 1) ? A : (xs ? As : Ar);
      const SC c1 = (xs ? fSR - fSS : fRR - fRS) * (xs ? qRS - qRR : qSS - qSR);
      const SC c2 = (xs ? fRS - fSS : fRR - fSR) * (xs ? qSR - qRR : qSS - qRS);
      gn[k] = sym ? (DT)2 * ((DT)A0 + (DT)c1) : (DT)A0 + (DT)c1 + (DT)c2;
      continue;
    }
    // scalars of the finish, loaded after the dot products: held across
    // them they cost registers (measured: int64 batch classes 2.3 %, the
    // n = 100 grid 1.7 % faster loaded here)
    const SC Frk = F[r * ldF + k], Fsk = F[s * ldF + k];
    const SC Fkr = Ft[r * ldF + k], Fks = Ft[s * ldF + k];
    const SC Qrk = Q[r * ldP + k], Qsk = Q[s * ldP + k];
    const SC Qkr = Qt[r * ldP + k], Qks = Qt[s * ldP + k];
    const SC Fkk = F[k * ldF + k], Qkk = Q[k * ldP + k];
    const SC a = Frk - Fsk, b = Qrk - Qsk, c = Fkr - Fks, e = Qkr - Qks;
    const DT gk = gc[k] - (DT)(a * b) - (DT)(c * e);
    for (int xi = lg; xi < 2; xi += (G == 1 ? 1 : 2)) {
      const bool xs = xi != 0;
      const SC fxx = xs ? fSS : fRR;   // F[x][x]
      const SC pxx = xs ? qRR : qSS;   // P'[x][x] = Q[xb][xb]
      const SC fxk = xs ? Fsk : Frk;   // F[x][k]
      const SC fkx = xs ? Fks : Fkr;   // F[k][x]
      const SC pxk = xs ? Qrk : Qsk;   // P'[x][k] = Q[xb][k]
      const SC pkx = xs ? Qkr : Qks;   // P'[k][x] = Q[k][xb]
      // exchanged columns: (F[x][r]-F[x][s]), (F[r][x]-F[s][x]),
      // (Q[xb][s]-Q[xb][r]), (Q[s][xb]-Q[r][xb])
      const SC fx_rs = xs ? fSR - fSS : fRR - fRS;
      const SC frs_x = xs ? fRS - fSS : fRR - fSR;
      const SC qxb_sr = xs ? qRS - qRR : qSS - qSR;
      const SC qsr_xb = xs ? qSR - qRR : qSS - qRS;
      const SC corr = (fxx - fxk - fkx + Fkk) * (pxx - pxk - pkx + Qkk);
      const SC sig = -fx_rs * e - frs_x * b + qxb_sr * c + qsr_xb * a;
      const SC Ax = (G > 1) ? A : (xs ? As : Ar);
      const SC Bx = (G > 1) ? B : (xs ? Bs : Br);
      const DT cross = sym ? (DT)2 * ((DT)Ax + (DT)Bx) : (DT)Ax + (DT)Bx;
      S.R[xi * n + k] = cross + (DT)sig - gk + (DT)corr;
    }
    if (lg == 0) {
      VO::put(S.vec, n, k, VO::pack(a, b, c, e));
      gn[k] = gk;
    }
  }
}

// ---------------------------------------------------------------------------
// Phase X from maintained products (plans with kProductM, int8 or int16 flows)
// ---------------------------------------------------------------------------
// These plans neither exchange rows and columns of P nor index M by
// location.  P keeps the walk's starting matrix P0 = D[p0][p0], and
// sigma[k] is the row of P0 that location k now holds (p = p0 o sigma), so
// Q[i][j] = P0[sigma[i]][sigma[j]]; a move (r s) exchanges sigma[r] and
// sigma[s] only.  The products are kept with their columns indexed by that
// label rather than by location: Mt[x][sigma[k]] = M[x][k] = F[x].Q[k] +
// F^T[x].Q^T[k].  A move changes Q only at the rows and columns r, s, and a
// label's column does not move with it: every entry takes the same rank-2
// update
//   Mt'[x][u] = Mt[x][u] - a_x b_j - c_x e_j,   j the location of label u
// before the move (with a, b, c, e the update vector of phase X), in place
// and with no exchange of columns.

// Mt from P0 at the start of a walk (sigma the identity): one dot product
// per entry (two when F or D is asymmetric; NOTR: the second over columns,
// element by element).  Mt[k][k] is g[k].
template <int NT, bool NOTR, typename DT, typename FE>
__device__ __forceinline__ void compute_m(const WalkSmem<DT, FE>& S, int32_t* Mt, int n, int ldF,
                                          int ldP, bool sym) {
  using C = Chunk<FE>;
  const int nc = (n + C::W - 1) / C::W, ldm = ld_m(n);
  for (int e = threadIdx.x; e < n * n; e += NT) {
    const int x = e / n, k = e - (e / n) * n;
    const auto* Fx = reinterpret_cast<const typename C::FV*>(S.F + x * ldF);
    const auto* Pk = reinterpret_cast<const typename C::QV*>(S.P + k * ldP);
    const auto* Ftx = reinterpret_cast<const typename C::FV*>(S.Ft + x * ldF);
    const auto* Ptk = reinterpret_cast<const typename C::QV*>(S.Pt + k * ldP);
    int acc = 0;
    for (int c = 0; c < nc; ++c) {
      acc = C::dot(Fx[c], Pk[c], acc);
      if (!NOTR && !sym) acc = C::dot(Ftx[c], Ptk[c], acc);
    }
    if (NOTR && !sym)
      for (int j = 0; j < n; ++j) acc += (int)S.F[j * ldF + x] * (int)S.P[j * ldP + k];
    Mt[x * ldm + k] = sym ? 2 * acc : acc;
  }
}

// Phase X of move (r, s) from Mt (pre-move): one thread per index k writes
// the update vector of k, also as the operands of phase_m_update: by index
// the row operand (-a_k, -c_k) in vw, by label the column operand (b_k, e_k)
// in vwu at sigma[k] (int8 flows: bytes (-a, -c, 0, 0) and the packed word
// (b, e, a, c), one dp4a; int16 flows whose differences fit (d16): int16
// (-a, -c) and bytes (b, e, 0, 0), one dp2a; other int16 flows: the int32
// pairs (a, c) and (b, e)); and, for k outside {r, s}, the recomputed
// deltas of the
// pairs {r, k} and {s, k}, whose dot products are the entries
//   F[r].Q[k] + F^T[r].Q^T[k] = M[r][k],  F[k].Q[s] + F^T[k].Q^T[s] = M[k][s]
// (and the same with r, s exchanged); the threads of k = r and k = s write
// g'[r] = M'[r][r] = M[r][s] - a_r b_s - c_r e_s and g'[s] likewise.  Q is
// read from P0 through sigma.  The finish is the one of phase_x.
template <typename DT, typename FE, int NT, bool NOTR, typename VO>
__device__ __forceinline__ void phase_m_prep(const WalkSmem<DT, FE>& S, const int32_t* Mt,
                                             int32_t* vw, int32_t* vwu, const int32_t* sigma,
                                             DT* gn, int n, int ldF, int ldP, int r, int s,
                                             bool d16) {
  const FE* F = S.F;
  const FE* Ft = S.Ft;
  const int8_t* P0 = S.P;
  const int8_t* P0t = S.Pt;
  const int ldm = ld_m(n);
  const int ur = sigma[r], us = sigma[s];  // P0 rows of locations r and s
  const int8_t* Qr = P0 + ur * ldP;         // Q[r][j] = Qr[sigma[j]]
  const int8_t* Qs = P0 + us * ldP;
  // Q^T[r][j] = Qtr[sigma[j] * qs] (NOTR: column ur of P0)
  const int8_t* Qtr = NOTR ? P0 + ur : P0t + ur * ldP;
  const int8_t* Qts = NOTR ? P0 + us : P0t + us * ldP;
  const int qs = NOTR ? ldP : 1;
  for (int k = threadIdx.x; k < n; k += NT) {
    const int uk = sigma[k];
    const int Frk = F[r * ldF + k], Fsk = F[s * ldF + k];
    const int Fkr = NOTR ? F[k * ldF + r] : Ft[r * ldF + k];
    const int Fks = NOTR ? F[k * ldF + s] : Ft[s * ldF + k];
    const int Qrk = Qr[uk], Qsk = Qs[uk];
    const int Qkr = Qtr[uk * qs], Qks = Qts[uk * qs];
    const int a = Frk - Fsk, b = Qrk - Qsk, c = Fkr - Fks, e = Qkr - Qks;
    const typename VO::V v = VO::pack(a, b, c, e);
    VO::put(S.vec, n, k, v);
    if constexpr (sizeof(FE) == 1) {
      // the int8 path keeps every difference within +-127: -a, -c fit a byte
      vw[k] = (int)(((uint32_t)(-a) & 0xffu) | (((uint32_t)(-c) & 0xffu) << 8));
      vwu[uk] = v.x;
    } else if (d16) {
      vw[k] = (int)(((uint32_t)(-a) & 0xffffu) | ((uint32_t)(-c) << 16));
      vwu[uk] = (int)(((uint32_t)b & 0xffu) | (((uint32_t)e & 0xffu) << 8));
    } else {
      reinterpret_cast<int2*>(vw)[k] = make_int2(a, c);
      reinterpret_cast<int2*>(vwu)[uk] = make_int2(b, e);
    }
    if (k == r || k == s) {
      // g'[x] = M[x][xb] - c_x e_xb - a_x b_xb, xb the other of r, s
      const int uxb = k == s ? ur : us;
      const int exb = Qtr[uxb * qs] - Qts[uxb * qs];
      const int bxb = Qr[uxb] - Qs[uxb];
      gn[k] = (DT)Mt[k * ldm + uxb] - (DT)(c * exb) - (DT)(a * bxb);
      continue;
    }
    const int fRR = F[r * ldF + r], fRS = F[r * ldF + s];
    const int fSR = F[s * ldF + r], fSS = F[s * ldF + s];
    const int qRR = Qr[ur], qRS = Qr[us];
    const int qSR = Qs[ur], qSS = Qs[us];
    const int Fkk = F[k * ldF + k], Qkk = P0[uk * ldP + uk];
    const DT gk = (DT)Mt[k * ldm + uk] - (DT)(a * b) - (DT)(c * e);
#pragma unroll
    for (int xi = 0; xi < 2; ++xi) {
      const bool xs = xi != 0;
      const int fxx = xs ? fSS : fRR;   // F[x][x]
      const int pxx = xs ? qRR : qSS;   // P'[x][x] = Q[xb][xb]
      const int fxk = xs ? Fsk : Frk;   // F[x][k]
      const int fkx = xs ? Fks : Fkr;   // F[k][x]
      const int pxk = xs ? Qrk : Qsk;   // P'[x][k] = Q[xb][k]
      const int pkx = xs ? Qkr : Qks;   // P'[k][x] = Q[k][xb]
      const int fx_rs = xs ? fSR - fSS : fRR - fRS;
      const int frs_x = xs ? fRS - fSS : fRR - fSR;
      const int qxb_sr = xs ? qRS - qRR : qSS - qSR;
      const int qsr_xb = xs ? qSR - qRR : qSS - qRS;
      const int corr = (fxx - fxk - fkx + Fkk) * (pxx - pxk - pkx + Qkk);
      const int sig = -fx_rs * e - frs_x * b + qxb_sr * c + qsr_xb * a;
      const int Ax = Mt[(xs ? s : r) * ldm + uk];  // M[x][k]
      const int Bx = Mt[k * ldm + (xs ? ur : us)];  // M[k][xb]
      S.R[xi * n + k] = (DT)Ax + (DT)Bx + (DT)sig - gk + (DT)corr;
    }
  }
}

// A thread's share of the Mt update: one group of 4 consecutive unit columns
// (16-byte loads and stores) on every rows-th row from x0.  Fixed per walk.
struct MShare {
  int g, x0, rows;
};

__device__ __forceinline__ MShare m_share(int n, int nt) {
  const int gpr = ld_m(n) / 4;  // groups per row
  const int rows = nt / gpr;     // rows per pass: every thread below rows * gpr has a group
  return MShare{(int)threadIdx.x % gpr, (int)threadIdx.x / gpr, rows};
}

// Mt after move (r, s), in place, with the update operands of phase_m_prep:
//   Mt'[x][u] -= (a_x, c_x) . (b_j, e_j),  j the location of label u before
// the move: one dp4a (int8 flows) or dp2a (int16 flows, d16) of the row
// operand (-a_x, -c_x) with the column operand, accumulating into the entry;
// two multiply-adds of int32 pairs for the other int16 flows.  Runs after
// the owner pass, which does not read Mt;
// phase_m_prep of this move read it before the barrier that precedes the
// owner pass, and the next one reads it after the next arg-min's barrier.
// Columns past n are padding.
template <typename FE>
__device__ __forceinline__ void phase_m_update(int32_t* Mt, const int32_t* vw,
                                               const int32_t* vwu, int n, MShare sh, bool d16) {
  if (sh.x0 >= sh.rows) return;
  const int ldm = ld_m(n);
  if (sizeof(FE) == 1 || d16) {
    const int4 w = reinterpret_cast<const int4*>(vwu)[sh.g];
    auto upd = [&](int u, int4 m) {
      if constexpr (sizeof(FE) == 1) {
        m.x = __dp4a(u, w.x, m.x);
        m.y = __dp4a(u, w.y, m.y);
        m.z = __dp4a(u, w.z, m.z);
        m.w = __dp4a(u, w.w, m.w);
      } else {
        m.x = __dp2a_lo(u, w.x, m.x);
        m.y = __dp2a_lo(u, w.y, m.y);
        m.z = __dp2a_lo(u, w.z, m.z);
        m.w = __dp2a_lo(u, w.w, m.w);
      }
      return m;
    };
    int x = sh.x0;
    if constexpr (sizeof(FE) == 2) {
      // two rows per step (measured: int16 batch512 2700.6 -> 2673.8 ms per
      // step; the int8 plans 0.3-0.4 % slower, so they keep one)
      for (; x + sh.rows < n; x += 2 * sh.rows) {
        const int x1 = x + sh.rows;
        const int u0 = vw[x], u1 = vw[x1];
        int4* M0 = reinterpret_cast<int4*>(Mt + x * ldm) + sh.g;
        int4* M1 = reinterpret_cast<int4*>(Mt + x1 * ldm) + sh.g;
        const int4 m0 = *M0, m1 = *M1;
        *M0 = upd(u0, m0);
        *M1 = upd(u1, m1);
      }
    }
    for (; x < n; x += sh.rows) {
      int4* Mx = reinterpret_cast<int4*>(Mt + x * ldm) + sh.g;
      *Mx = upd(vw[x], *Mx);
    }
  } else {
    // (b, e) of the group's 4 labels
    const int4 w0 = reinterpret_cast<const int4*>(vwu)[2 * sh.g];
    const int4 w1 = reinterpret_cast<const int4*>(vwu)[2 * sh.g + 1];
    for (int x = sh.x0; x < n; x += sh.rows) {
      const int2 ac = reinterpret_cast<const int2*>(vw)[x];
      int4* Mx = reinterpret_cast<int4*>(Mt + x * ldm) + sh.g;
      int4 m = *Mx;
      m.x -= ac.x * w0.x + ac.y * w0.y;
      m.y -= ac.x * w0.z + ac.y * w0.w;
      m.z -= ac.x * w1.x + ac.y * w1.y;
      m.w -= ac.x * w1.z + ac.y * w1.w;
      *Mx = m;
    }
  }
}

// Exchange rows and columns r, s of P (and P^T) and p[r], p[s], so that
// P'[i][j] = P[s(i)][s(j)] with s the transposition (r s).  Column entries of
// the other rows: one thread per (matrix, row); rows r and s: 4-byte words by
// the last warp (lanes 0-15 for P, 16-31 for P^T), whose lanes then exchange
// the entries r and s inside those two rows.
template <int NT, typename PE>
__device__ __forceinline__ void swap_rs(PE* P, PE* Pt, int32_t* perm, int n, int ldP, bool symD,
                                        int r, int s) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    const int32_t t = perm[r];
    perm[r] = perm[s];
    perm[s] = t;
  }
  const int mats = symD ? 1 : 2;
  for (int c = tid; c < mats * n; c += NT) {
    const int j = c < n ? c : c - n;
    if (j == r || j == s) continue;
    PE* Pj = (c < n ? P : Pt) + j * ldP;
    const PE t = Pj[r];
    Pj[r] = Pj[s];
    Pj[s] = t;
  }
  if (tid >= NT - 32) {
    const int lane = tid & 31, m = lane >> 4, l = lane & 15;
    if (m < mats) {
      PE* M = m ? Pt : P;
      int32_t* Mr = reinterpret_cast<int32_t*>(M + r * ldP);
      int32_t* Ms = reinterpret_cast<int32_t*>(M + s * ldP);
      const int words = (n * (int)sizeof(PE) + 3) / 4;
      for (int w = l; w < words; w += 16) {
        const int32_t a = Mr[w];
        Mr[w] = Ms[w];
        Ms[w] = a;
      }
    }
    __syncwarp();
    if (l == 0 && m < mats) {
      PE* M = m ? Pt : P;
      PE* Rr = M + r * ldP;
      PE* Rs = M + s * ldP;
      PE t = Rr[r]; Rr[r] = Rr[s]; Rr[s] = t;
      t = Rs[r]; Rs[r] = Rs[s]; Rs[s] = t;
    }
  }
}

// ---------------------------------------------------------------------------
// the walk kernel
// ---------------------------------------------------------------------------
constexpr int min_blocks(int nt) { return nt <= 128 ? 4 : nt <= 256 ? 2 : 1; }

// Pairs are handed out by rows: row u holds the pairs (u, v), v > u, and
// gets c_u = ceil((n - 1 - u) / MAXPT) threads, in row-major order.  Its
// thread j owns either the run v = u + 1 + j MAXPT + i (contiguous), or
// v = u + 1 + j + i c_u (interleaved: at each slot the threads of a row read
// consecutive entries of the per-index arrays, free of shared-memory bank
// conflicts for 16-byte entries), i = 0, 1, ... (at most MAXPT).  The host
// checks that every row segment (one per thread) has a thread.
__host__ __device__ inline int row_segments(int n, int maxpt) {
  int nseg = 0;
  for (int u = 0; u < n - 1; ++u) nseg += (n - 1 - u + maxpt - 1) / maxpt;
  return nseg;
}

// The interleaved layout where it measured faster: 16-byte per-index entries
// (int16 flows), up to 512 threads (at 1024 the extra registers spill).
template <typename FE, int NT>
__host__ __device__ constexpr bool interleaved() { return sizeof(FE) == 2 && NT <= 512; }

struct Segment {
  int su, sv, sk, slen;  // pairs (su, sv + i sk), i < slen
  int wlen;              // most slots in the warp
};

template <int MAXPT, bool INTERLEAVE>
__device__ __forceinline__ Segment make_segment(int n) {
  Segment g{0, 1, 1, 0, 0};
  const int tid = threadIdx.x;
  int t0 = 0;
  for (int u = 0; u < n - 1; ++u) {
    const int len = n - 1 - u;
    const int ns = (len + MAXPT - 1) / MAXPT;
    if (tid >= t0 && tid < t0 + ns) {
      const int j = tid - t0;
      g.su = u;
      if (INTERLEAVE) {
        g.sv = u + 1 + j;
        g.sk = ns;
        g.slen = (len - j + ns - 1) / ns;  // at most MAXPT
      } else {
        g.sv = u + 1 + j * MAXPT;
        g.slen = min(MAXPT, len - j * MAXPT);
      }
    }
    t0 += ns;
  }
  g.wlen = __reduce_max_sync(kFull, g.slen);
  return g;
}

template <typename DT, typename FE, int NT, int MAXPT, int STORE>
__device__ __forceinline__ WalkSmem<DT, FE> smem_views(unsigned char* smem, const InstArgs& I,
                                                       unsigned char* ws, size_t p_off) {
  using PE = typename Elem<FE>::P;
  const SmemLayout L = smem_layout(I.n, I.ldF, (int)sizeof(FE), I.ldP, I.symF, I.symD,
                                   (int)sizeof(DT), NT * MAXPT, STORE);
  WalkSmem<DT, FE> S;
  if (STORE & kGlobalFlow) {
    S.F = const_cast<FE*>(reinterpret_cast<const FE*>(I.F));
    S.Ft = const_cast<FE*>(reinterpret_cast<const FE*>(I.Ft));
  } else {
    S.F = reinterpret_cast<FE*>(smem + L.offF);
    S.Ft = (I.symF || (STORE & kNoTransposed)) ? S.F : reinterpret_cast<FE*>(smem + L.offFt);
  }
  if (STORE & kGlobalP) {
    S.P = reinterpret_cast<PE*>(ws + p_off);
    S.Pt = I.symD ? S.P : S.P + (size_t)I.n * I.ldP;
  } else {
    S.P = reinterpret_cast<PE*>(smem + L.offP);
    S.Pt = (I.symD || (STORE & kNoTransposed)) ? S.P : reinterpret_cast<PE*>(smem + L.offPt);
  }
  // workspace: deltas (NT * MAXPT x DT), then tabu stamps (NT * MAXPT x int32)
  S.tabu = (STORE & kGlobalDelta)
               ? reinterpret_cast<int32_t*>(ws + (size_t)NT * MAXPT * sizeof(DT))
               : reinterpret_cast<int32_t*>(smem + L.offTabu);
  S.vec = smem + L.offVec;
  S.R = reinterpret_cast<DT*>(smem + L.offR);
  S.g0 = reinterpret_cast<DT*>(smem + L.offG0);
  S.g1 = reinterpret_cast<DT*>(smem + L.offG1);
  S.perm = reinterpret_cast<int32_t*>(smem + L.offPerm);
  S.best = reinterpret_cast<int32_t*>(smem + L.offBest);
  S.redD = reinterpret_cast<DT*>(smem + L.offRedD);
  S.redK = reinterpret_cast<uint32_t*>(smem + L.offRedK);
  S.sum = reinterpret_cast<int64_t*>(smem + L.offSum);
  S.M = (STORE & kProductM) ? reinterpret_cast<int32_t*>(smem + L.offM) : nullptr;
  return S;
}

// F (and F^T) into shared memory (rows are whole 16-byte vectors, zero
// padded); P (and P^T) zeroed so their padding columns stay zero.  Ends with
// a barrier.
template <typename DT, typename FE, int NT, int STORE>
__device__ __forceinline__ void load_instance(const WalkSmem<DT, FE>& S, const InstArgs& I) {
  const int tid = threadIdx.x;
  const int nvec = I.n * I.ldF * (int)sizeof(FE) / 16;
  const int4* gF = reinterpret_cast<const int4*>(I.F);
  int4* sF = reinterpret_cast<int4*>(S.F);
  if (!(STORE & kGlobalFlow))
    for (int i = tid; i < nvec; i += NT) sF[i] = gF[i];
  if (!I.symF && !(STORE & (kGlobalFlow | kNoTransposed))) {
    const int4* gFt = reinterpret_cast<const int4*>(I.Ft);
    int4* sFt = reinterpret_cast<int4*>(S.Ft);
    for (int i = tid; i < nvec; i += NT) sFt[i] = gFt[i];
  }
  const int pvec = I.n * I.ldP * (int)sizeof(typename Elem<FE>::P) / 16;
  int4* sP = reinterpret_cast<int4*>(S.P);
  for (int i = tid; i < pvec; i += NT) sP[i] = make_int4(0, 0, 0, 0);
  if (!I.symD && !(STORE & kNoTransposed)) {
    int4* sPt = reinterpret_cast<int4*>(S.Pt);
    for (int i = tid; i < pvec; i += NT) sPt[i] = make_int4(0, 0, 0, 0);
  }
  __syncthreads();
}

// The deltas of a thread's slots: registers, or the CTA's workspace.
template <typename DT, int NT, int MAXPT, bool GLOBAL>
struct DeltaSlots;

template <typename DT, int NT, int MAXPT>
struct DeltaSlots<DT, NT, MAXPT, false> {
  DT v[MAXPT];
  __device__ __forceinline__ explicit DeltaSlots(unsigned char*) {}
  __device__ __forceinline__ DT get(int i) const { return v[i]; }
  __device__ __forceinline__ void set(int i, DT x) { v[i] = x; }
};

template <typename DT, int NT, int MAXPT>
struct DeltaSlots<DT, NT, MAXPT, true> {
  DT* p;  // slot i at p[i * NT]
  __device__ __forceinline__ explicit DeltaSlots(unsigned char* ws)
      : p(reinterpret_cast<DT*>(ws) + threadIdx.x) {}
  __device__ __forceinline__ DT get(int i) const { return p[(size_t)i * NT]; }
  __device__ __forceinline__ void set(int i, DT x) { p[(size_t)i * NT] = x; }
};

// One whole walk: start permutation, P, Eq. 1, the initial deltas, the 2opt
// descent, the tabu iterations and the outputs (row `row`).  `wid` is the
// walk id of the random draws; `start` a given start permutation or null.
// Starts and ends with every thread of the CTA together.
template <typename DT, typename FE, int NT, int MAXPT, int STORE>
__device__ __forceinline__ void run_walk(const WalkSmem<DT, FE>& S, const InstArgs& I,
                                         const Segment& seg, const SearchArgs& a, int row,
                                         uint32_t wid, const int32_t* start, unsigned char* ws) {
  const int n = I.n, ldF = I.ldF, ldP = I.ldP, tid = threadIdx.x, G = I.group;
  const bool sym = I.symF && I.symD;
  const bool warp0 = tid < 32;
  constexpr bool kInterleave = interleaved<FE, NT>();
  constexpr bool kNoTr = (STORE & kNoTransposed) != 0;
  // per-index vectors: the word-only form on the 6-slot products plan
  using VOsel = std::conditional_t<sizeof(FE) == 1 && (STORE & kProductM) != 0 && MAXPT == 6,
                                   VecOpsWord, VecOps<FE>>;
  const int su = seg.su, sv = seg.sv, slen = seg.slen, wlen = seg.wlen;
  const int sk = kInterleave ? seg.sk : 1;
  const int seg_sv = sv, seg_sk = sk;
  const uint32_t ukey = (uint32_t)su << 8;
  // slot of the pair (su, x), or -1 when this thread does not hold it
  auto slot_of = [&](int x) {
    const int d = x - sv;
    if (d < 0) return -1;
    const int q = d / sk;
    return q * sk == d && q < slen ? q : -1;
  };

  // Start permutation: given, or Fisher-Yates on stream 0.
  if (start) {
    for (int x = tid; x < n; x += NT) S.perm[x] = start[x];
  } else if (tid == 0) {
    for (int x = 0; x < n; ++x) S.perm[x] = x;
    Philox4 blk{};
    for (int i = n - 1; i >= 1; --i) {
      const uint32_t idx = (uint32_t)(n - 1 - i);
      if ((idx & 3u) == 0)
        blk = philox4x32_10(wid, 0u, idx >> 2, 0u, (uint32_t)a.seed, (uint32_t)(a.seed >> 32));
      const int j = (int)below(blk.v[idx & 3u], (uint32_t)(i + 1));
      const int32_t t = S.perm[i];
      S.perm[i] = S.perm[j];
      S.perm[j] = t;
    }
  }
  __syncthreads();

  // P = D[p][p] (and its transpose) gathered from global memory.
  using PE = typename Elem<FE>::P;
  const PE* Dg = reinterpret_cast<const PE*>(I.D);
  for (int c = tid; c < n * n; c += NT) {
    const int i = c / n, j = c - (c / n) * n;
    const PE v = Dg[(size_t)S.perm[i] * n + S.perm[j]];
    S.P[i * ldP + j] = v;
    if (!I.symD && !kNoTr) S.Pt[j * ldP + i] = v;
  }
  for (int x = tid; x < n; x += NT) S.best[x] = S.perm[x];
  __syncthreads();

  // Eq. 1, g, and the initial deltas of the owned pairs (Eq. 2, O(n) each).
  int64_t c0 = 0;
  for (int c = tid; c < n * n; c += NT) {
    const int i = c / n, j = c - (c / n) * n;
    c0 += (int64_t)S.F[i * ldF + j] * (int64_t)S.P[i * ldP + j];
  }
  c0 = block_sum<NT>(c0, S.sum);
  // maintained products (columns by unit), the update words by index and
  // by unit, and this thread's share of the update (held across the walk,
  // except at 1024 threads, whose 64 registers spill it)
  constexpr int kMW = m_words((int)sizeof(FE));
  int32_t* const Mt = S.M;
  int32_t* const vw = S.M ? S.M + n * ld_m(n) : nullptr;
  int32_t* const vwu = S.M ? vw + kMW * ld_m(n) : nullptr;
  int32_t* const sigma = S.M ? vwu + kMW * ld_m(n) : nullptr;
  [[maybe_unused]] const MShare msh = NT < 1024 ? m_share(n, NT) : MShare{};
  if constexpr ((STORE & kProductM) != 0) {
    for (int x = tid; x < n; x += NT) sigma[x] = x;
    compute_m<NT, kNoTr>(S, Mt, n, ldF, ldP, sym);
  }
  else
    compute_g<DT, FE, NT>(S, S.g0, n, ldF, ldP, sym, G);
  DeltaSlots<DT, NT, MAXPT, (STORE & kGlobalDelta) != 0> dl(ws);
  // owner pass form: the O(1) update everywhere with the rows r and s
  // handled inside the pass or after it (split), or one pass choosing per
  // slot between both values (fused).  Workspace slots are read and written
  // once (fused); register slots take the split pass (see kInlineRS).
  constexpr bool kSplitPass = !(STORE & kGlobalDelta);
#pragma unroll
  for (int i = 0; i < MAXPT; ++i) {
    dl.set(i, i < slen ? delta_serial<DT, FE, kNoTr>(S, n, ldF, ldP, sym, su, sv + i * sk)
                       : DeltaMax<DT>::v);
    S.tabu[i * NT + tid] = 0;
  }

  DT cur = (DT)c0;
  DT* gc = S.g0;
  DT* gn = S.g1;
  uint64_t h = 14695981039346656037ull, dh = h;
  int dmoves = 0;

  // Owners' pass after move (r, s): new deltas, then the scan for the next
  // iteration `nit` (tabu phase) or the next descent step.  Branch-free per
  // slot so the shared-memory loads of all slots are in flight together:
  // every slot takes the O(1) update, except the pairs (su, r) and (su, s)
  // of rows other than r and s, which take their recomputed rows.  The few
  // threads holding segments of rows r and s then recompute those and scan
  // again.
  // Tables of the other tabu criteria and of the frequency penalty, in the
  // CTA's workspace: loc_until[unit][location] (n x n), unit_until[unit] (n)
  // and applied[r][s] (n x n, the penalty's counts, row-major).  Addressed from the launch arguments when
  // used so that they hold no registers in the paper's own search.
  auto rule_tables = [&]() { return reinterpret_cast<int32_t*>(ws + a.rws_off); };
  auto applied = [&]() { return rule_tables() + n * n + n; };

  // With EXT (the other criteria or the frequency penalty in use) and a
  // penalty lambda, a non-improving pair is ranked by delta + lambda *
  // (times applied).
  auto update_and_scan = [&](auto ext, int r, int s, bool tabu, int nit, int stamp, DT ncur,
                             DT nbest, DT& bd, uint32_t& bk) {
    constexpr bool EXT = decltype(ext)::value;
    const int32_t* crow = EXT ? applied() + su * n : nullptr;
    using VO = VOsel;
    const void* vec = S.vec;
    const typename VO::U uu = VO::prep(VO::get(vec, n, su));
    const DT gr = gn[r], gs = gn[s];
    const bool tu = (su == r) | (su == s);        // every pair of the segment touches
    // admissible: not tabu (mark <= nit), or aspiring (ncur + d < nbest,
    // i.e. d < nbest - ncur, clamped where no delta can reach it)
    const int tlim = tabu ? nit : INT_MAX;
    DT lim = DeltaMin<DT>::v;
    if (!tabu) {
      lim = DeltaMax<DT>::v;
    } else if (a.aspiration) {
      const int64_t l = (int64_t)nbest - (int64_t)ncur;
      lim = l < (int64_t)DeltaMin<DT>::v ? DeltaMin<DT>::v : (DT)l;
    }
    auto rank = [&](DT d, int v) -> DT {
      if constexpr (EXT) return d >= 0 ? d + (DT)a.lambda * (DT)crow[v] : d;
      return d;
    };
    bd = DeltaMax<DT>::v;
    bk = kNoMove;
    [[maybe_unused]] int irs = -1;  // interleaved: slot of the pair (r, s), where held
    // interleaved: the slots' v are recomputed in each pass rather than held
    // across the iterations (which costs MAXPT registers)
    int sv = seg_sv, sk = seg_sk;
    if constexpr (kInterleave) asm volatile("" : "+r"(sv), "+r"(sk));
    const int ir = r - sv, is = s - sv;  // contiguous: slots of (su, r), (su, s) if held
    auto at_r = [&](int i) {
      if constexpr (kInterleave) return sv + i * sk == r;
      else return i == ir;
    };
    auto at_s = [&](int i) {
      if constexpr (kInterleave) return sv + i * sk == s;
      else return i == is;
    };
    if constexpr (kSplitPass) {
      // new deltas of the pairs (su, r) and (su, s) of other rows
      const DT xr = S.R[su] - gr, xs = S.R[n + su] - gs;
      // the pair (r, s) itself only changes sign
      DT nrs = 0;
      if (su == r) {
#pragma unroll
        for (int i = 0; i < MAXPT; ++i)
          if (at_s(i)) nrs = -dl.get(i);
      }
      // Rows r and s (tu): with int64 deltas or more than 4 slots their
      // owners take the recomputed value in this same pass, the row read
      // by those threads only (int64 batch classes 3.2 % faster; n = 100
      // grid, 256 x 24: 163.1 -> 156.6 ms, where a fused pass loading both
      // values for every slot had given 162.9 against the 180.8 of a
      // separate rescan; with the products form n = 50 asymmetric at 6
      // slots 7.91 -> 7.86 ms, n = 58 at 8 slots 7.90 -> 7.72 ms); with
      // int32 deltas and 4 slots they recompute and rescan their segments
      // after it (n = 30: 0.4 % faster than inline).
      constexpr bool kInlineRS = sizeof(DT) == 8 || MAXPT > 4;
      const int ubase = su == r ? 0 : n;
      const DT gu = su == r ? gr : gs;
#pragma unroll
      for (int i = 0; i < MAXPT; ++i) {
        if (i >= wlen) break;
        const bool valid = i < slen;
        const int vi = sv + i * sk;
        const int v = valid ? vi : sv;
        DT d = VO::update(uu, VO::get(vec, n, v), dl.get(i));
        d = at_r(i) ? xr : at_s(i) ? xs : d;
        bool isrs = false;
        if constexpr (kInlineRS) {
          isrs = (su == r) & at_s(i);
          if (tu) d = isrs ? nrs : S.R[ubase + v] - gu;
          if constexpr (kInterleave) {
            if (valid & isrs) irs = i;
          }
        }
        dl.set(i, d);
        const int tb = isrs ? stamp : S.tabu[i * NT + tid];
        const DT sc = rank(d, v);
        if (valid && (tb <= tlim || d < lim) && sc < bd) {
          bd = sc;
          bk = ukey | (uint32_t)v;
        }
      }
      if (!kInlineRS && tu) {
        // rows r and s: every pair recomputed, then scanned again; the pair
        // just applied carries its new mark
        bd = DeltaMax<DT>::v;
        bk = kNoMove;
        // int32 deltas, 4 slots here: slen differs between the
        // lanes, and the slots past it are predicated off rather than left
        // by a branch (measured faster)
#pragma unroll
        for (int i = 0; i < MAXPT; ++i) {
          const bool valid = i < slen;
          const int vi = sv + i * sk;
          const int v = valid ? vi : sv;
          const bool isrs = (su == r) & at_s(i);
          const DT dn = isrs ? nrs : S.R[ubase + v] - gu;
          const DT d = valid ? dn : dl.get(i);
          dl.set(i, d);
          if constexpr (kInterleave) {
            if (valid & isrs) irs = i;
          }
          const int tb = isrs ? stamp : S.tabu[i * NT + tid];
          const DT sc = rank(d, v);
          if (valid && (tb <= tlim || d < lim) && sc < bd) {
            bd = sc;
            bk = ukey | (uint32_t)v;
          }
        }
      }
    } else {
      // one pass, each slot choosing between its update and its recomputed
      // row
      const int ubase = su == r ? 0 : n;
      const DT gu = su == r ? gr : gs;
#pragma unroll
      for (int i = 0; i < MAXPT; ++i) {
        if (i >= wlen) break;
        const bool valid = i < slen;
        const int vi = sv + i * sk;
        const int v = valid ? vi : sv;
        const bool tvr = at_r(i), tv = tvr | at_s(i);
        const int idx = tu ? ubase + v : (tvr ? 0 : n) + su;  // in range for any v, su
        const DT rv = S.R[idx];
        const int tbl = S.tabu[i * NT + tid];
        const DT gx = tu ? gu : (tvr ? gr : gs);
        DT d = dl.get(i);
        const DT o1 = VO::update(uu, VO::get(vec, n, v), d);
        const bool isrs = (su == r) & at_s(i);
        d = isrs ? -d : (tu | tv) ? rv - gx : o1;
        dl.set(i, d);
        if constexpr (kInterleave) {
          if (valid & isrs) irs = i;
        }
        const int tb = isrs ? stamp : tbl;
        const DT sc = rank(d, v);
        if (valid && (tb <= tlim || d < lim) && sc < bd) {
          bd = sc;
          bk = ukey | (uint32_t)v;
        }
      }
    }
    if constexpr (kInterleave) {
      if (tabu && irs >= 0) S.tabu[irs * NT + tid] = stamp;
    } else {
      if (tabu && su == r && s >= sv && s < sv + slen) S.tabu[(s - sv) * NT + tid] = stamp;
    }
  };

  // The move's exchange: rows and columns r, s of P (and P^T) and p[r],
  // p[s]; with the maintained products p[r], p[s] and sigma[r], sigma[s]
  // only (P stays P0).
  auto apply_move = [&](int r, int s) {
    if constexpr ((STORE & kProductM) != 0) {
      if (tid == 0) {
        int32_t t = S.perm[r];
        S.perm[r] = S.perm[s];
        S.perm[s] = t;
        t = sigma[r];
        sigma[r] = sigma[s];
        sigma[s] = t;
      }
    } else {
      swap_rs<NT>(S.P, S.Pt, S.perm, n, ldP, I.symD, r, s);
    }
  };

  // Phase X of move (r, s): from the maintained products (kProductM), or
  // by dot products over the rows of F and P.
  auto phase_x_any = [&](int r, int s) {
    if constexpr ((STORE & kProductM) != 0)
      phase_m_prep<DT, FE, NT, kNoTr, VOsel>(S, Mt, vw, vwu, sigma, gn, n, ldF, ldP, r, s,
                                              I.diff16 != 0);
    else
      phase_x<DT, FE, NT>(S, gc, gn, n, ldF, ldP, sym, G, r, s);
  };

  // ---- 2opt descent (Section 4.1): best move while it improves.
  if (a.descend) {
    // A descent strictly lowers the cost at every move, so it ends; the
    // cap only bounds the kernel's run time on any input.
    const int cap = a.max_descent >= 0 ? a.max_descent : kDescentCap;
    DT bd = DeltaMax<DT>::v;
    uint32_t bk = kNoMove;
#pragma unroll
    for (int i = 0; i < MAXPT; ++i)
      if (i < slen && dl.get(i) < bd) {
        bd = dl.get(i);
        bk = ukey | (uint32_t)(sv + i * sk);
      }
    for (;;) {
      if (dmoves >= cap) break;
      block_argmin<DT, NT>(bd, bk, S.redD, S.redK);
      if (bk == kNoMove || bd >= 0) break;
      const int r = (int)(bk >> 8), s = (int)(bk & 0xffu);
      cur += bd;
      ++dmoves;
      if (warp0) dh = fnv_step(dh, r, s);
      phase_x_any(r, s);
      __syncthreads();
      update_and_scan(std::false_type{}, r, s, false, 0, 0, cur, cur, bd, bk);
      apply_move(r, s);
      if constexpr ((STORE & kProductM) != 0) {
        // Mt after the move (read by the next phase X, after the next
        // arg-min's barrier); after the owner pass, so that each thread's
        // candidate is ready first (asym50 10.14 -> 10.04 ms per step)
        phase_m_update<FE>(Mt, vw, vwu, n, NT < 1024 ? msh : m_share(n, NT), I.diff16 != 0);
      }
      DT* t = gc; gc = gn; gn = t;
    }
    __syncthreads();
    for (int x = tid; x < n; x += NT) S.best[x] = S.perm[x];
  }

  // ---- tabu search (Sections 4.3, 4.4).
  // frequency memory of this walk (Section 4.3): zeroed here, then the owner
  // of each applied move adds one at [s][r]
  int32_t* fq = a.freq ? a.freq + (size_t)row * a.p_stride * a.p_stride : nullptr;
  if (fq)
    for (int c = tid; c < a.p_stride * a.p_stride; c += NT) fq[c] = 0;
  // The other criteria keep each pair's mark ("until") in S.tabu as the
  // paper's does: only the pairs touching r or s change it at a move.
  const bool rules = a.iters > 0 && (a.crit != 0 || a.lambda != 0);
  if (rules) {
    int32_t* t = rule_tables();
    for (int c = tid; c < 2 * n * n + n; c += NT) t[c] = 0;
  }
  if (fq || rules) __syncthreads();
  // locations of the move's units before it: S.sum's first two words (the
  // block sum is done by now); written after the arg-min, read after the
  // next barrier, before swap_rs can have moved them
  int32_t* moved_from = reinterpret_cast<int32_t*>(S.sum);
  int tmin = a.tmin, tmax = a.tmax, period = a.period;
  if (a.tenure_per_n) {
    tmin = max(1, a.tmin * n / 100);
    tmax = max(tmin, (a.tmax * n + 99) / 100);
    period = a.period * n / 100;
  }
  DT best = cur;
  int best_iter = 0, status = 0, done = 0;
  bool copy_pending = false;
  int tenure = 0, tleft = 1;  // period > 0: a new tenure when tleft reaches 0
  uint32_t tdraw = 0;
  DT bd = DeltaMax<DT>::v;
  uint32_t bk = kNoMove;
  if (a.iters > 0) {
#pragma unroll
    for (int i = 0; i < MAXPT; ++i) {
      const DT d = dl.get(i);
      const bool adm = S.tabu[i * NT + tid] <= 1 || (a.aspiration && cur + d < best);
      if (i < slen && adm && d < bd) {
        bd = d;
        bk = ukey | (uint32_t)(sv + i * sk);
      }
    }
  }
  // The iterations; EXT adds the other criteria and the penalty, so that
  // the paper's own search runs a loop without their code.
  auto tabu_loop = [&](auto ext) {
    constexpr bool EXT = decltype(ext)::value;
    for (int it = 1; it <= a.iters; ++it) {
      block_argmin<DT, NT>(bd, bk, S.redD, S.redK);
      if (copy_pending) {  // p after the previous iteration's move
        for (int x = tid; x < n; x += NT) S.best[x] = S.perm[x];
        copy_pending = false;
      }
      if (bk == kNoMove) {
        status = 1;
        break;
      }
      const int r = (int)(bk >> 8), s = (int)(bk & 0xffu);
      if constexpr (EXT) {
        // bd is the move's rank; with the penalty a non-improving rank
        // holds lambda * applied[r][s] on top of the delta
        if (a.lambda != 0 && bd >= 0) bd -= (DT)a.lambda * (DT)applied()[r * n + s];
        if (a.crit != 0 && tid == 0) {
          moved_from[0] = S.perm[r];
          moved_from[1] = S.perm[s];
        }
      }
      cur += bd;
      done = it;
      if (warp0) h = fnv_step(h, r, s);
      if (cur < best) {
        best = cur;
        best_iter = it;
        copy_pending = true;
      }
      if (period > 0 && --tleft == 0) {  // it = 1, period + 1, ...
        const uint32_t x = walk_draw(a.seed, wid, 1u, tdraw++);
        tenure = tmin + (int)below(x, (uint32_t)(tmax - tmin + 1));
        tleft = period;
      }
      phase_x_any(r, s);
      __syncthreads();
      int stamp = it + tenure;
      const bool owner =
          su == r && (kInterleave ? slot_of(s) >= 0 : s >= sv && s < sv + slen);
      if (period == 0 && (owner || (EXT && a.crit != 0))) {
        // the paper's rule: a fresh tenure per move, drawn by the owner only
        // (by every thread when the other criteria restamp touching pairs)
        const uint32_t x = walk_draw(a.seed, wid, 1u, (uint32_t)(it - 1));
        stamp = it + tmin + (int)below(x, (uint32_t)(tmax - tmin + 1));
      }
      if constexpr (EXT) {
        if (a.crit != 0) {
          // New marks of the pairs touching r or s, read through this
          // move's own marks (units r, s leave locations pr, ps), which
          // thread 0 also stores for the next iterations.
          int32_t* loc_until = rule_tables();
          int32_t* unit_until = loc_until + n * n;
          const int pr = moved_from[0], ps = moved_from[1];
          auto loc_mark = [&](int u, int l) {
            return (u == r && l == pr) || (u == s && l == ps) ? stamp : loc_until[u * n + l];
          };
          auto unit_mark = [&](int u) { return u == r || u == s ? stamp : unit_until[u]; };
          auto after = [&](int x) { return x == r ? ps : x == s ? pr : S.perm[x]; };
          auto mark = [&](int u, int v) {
            return a.crit == 1 ? min(loc_mark(u, after(v)), loc_mark(v, after(u)))
                               : max(unit_mark(u), unit_mark(v));
          };
          if (su == r || su == s) {
            for (int i = 0; i < slen; ++i) S.tabu[i * NT + tid] = mark(su, sv + i * sk);
          } else if constexpr (kInterleave) {
            const int ir = slot_of(r), is = slot_of(s);
            if (ir >= 0) S.tabu[ir * NT + tid] = mark(su, r);
            if (is >= 0) S.tabu[is * NT + tid] = mark(su, s);
          } else {
            if (r >= sv && r < sv + slen) S.tabu[(r - sv) * NT + tid] = mark(su, r);
            if (s >= sv && s < sv + slen) S.tabu[(s - sv) * NT + tid] = mark(su, s);
          }
          if (tid == 0) {
            loc_until[r * n + pr] = stamp;
            loc_until[s * n + ps] = stamp;
            unit_until[r] = stamp;
            unit_until[s] = stamp;
          }
        }
        // read above by every thread before the barrier
        if (a.lambda != 0 && owner) applied()[r * n + s] += 1;
      }
      update_and_scan(ext, r, s, true, it + 1, stamp, cur, best, bd, bk);
      if (fq && owner) atomicAdd(fq + s * a.p_stride + r, 1);
      apply_move(r, s);
      if constexpr ((STORE & kProductM) != 0) {
        // Mt after the move (read by the next phase X, after the next
        // arg-min's barrier); after the owner pass, so that each thread's
        // candidate is ready first (asym50 10.14 -> 10.04 ms per step)
        phase_m_update<FE>(Mt, vw, vwu, n, NT < 1024 ? msh : m_share(n, NT), I.diff16 != 0);
      }
      DT* t = gc; gc = gn; gn = t;
    }
  };
  if (rules)
    tabu_loop(std::true_type{});
  else
    tabu_loop(std::false_type{});
  __syncthreads();
  if (copy_pending)
    for (int x = tid; x < n; x += NT) S.best[x] = S.perm[x];
  __syncthreads();

  // ---- outputs
  if (a.best_p)
    for (int x = tid; x < n; x += NT) a.best_p[(size_t)row * a.p_stride + x] = S.best[x];
  if (tid == 0) {
    a.best_cost[row] = (int64_t)best;
    if (a.final_cost) a.final_cost[row] = (int64_t)cur;
    if (a.best_iter) a.best_iter[row] = best_iter;
    if (a.iters_done) a.iters_done[row] = done;
    if (a.status) a.status[row] = status;
    if (a.descent_moves) a.descent_moves[row] = dmoves;
    if (a.hash) a.hash[row] = h;
    if (a.descent_hash) a.descent_hash[row] = dh;
  }
  __syncthreads();
}

// Walks of one instance; CTAs loop over walks.
template <typename DT, typename FE, int NT, int MAXPT, int STORE>
__global__ void __launch_bounds__(NT, min_blocks(NT)) walk_kernel(const WalkArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* ws = a.ws ? a.ws + a.ws_stride * blockIdx.x : nullptr;
  const WalkSmem<DT, FE> S = smem_views<DT, FE, NT, MAXPT, STORE>(smem, a.inst, ws, a.s.p_off);
  const Segment seg = make_segment<MAXPT, interleaved<FE, NT>()>(a.inst.n);
  load_instance<DT, FE, NT, STORE>(S, a.inst);
  for (int w = blockIdx.x; w < a.walks; w += gridDim.x) {
    const int wi = a.walk_offset + w;
    run_walk<DT, FE, NT, MAXPT, STORE>(S, a.inst, seg, a.s, wi, a.s.walk_base + (uint32_t)wi,
                                       a.starts ? a.starts + (size_t)wi * a.inst.n : nullptr,
                                       ws);
  }
}

// Walks of many instances; CTAs take (instance, walk) items from a counter
// and reload F when the instance changes.
template <typename DT, typename FE, int NT, int MAXPT, int STORE>
__global__ void __launch_bounds__(NT, min_blocks(NT)) batch_kernel(const BatchArgs b) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int item_s;
  unsigned char* ws = b.ws ? b.ws + b.ws_stride * blockIdx.x : nullptr;
  int cur_inst = -1;
  WalkSmem<DT, FE> S{};
  Segment seg{};
  InstArgs I{};
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(b.counter, 1);
    __syncthreads();
    const int item = item_s;
    __syncthreads();
    if (item >= b.items) break;
    const int inst = b.item_inst[item], w = b.item_walk[item];
    if (inst != cur_inst) {
      I = b.insts[inst];
      S = smem_views<DT, FE, NT, MAXPT, STORE>(smem, I, ws, b.s.p_off);
      seg = make_segment<MAXPT, interleaved<FE, NT>()>(I.n);
      load_instance<DT, FE, NT, STORE>(S, I);
      cur_inst = inst;
    }
    run_walk<DT, FE, NT, MAXPT, STORE>(S, I, seg, b.s, b.row_base[inst] + w,
                                       b.s.walk_base + (uint32_t)w, nullptr, ws);
  }
}

using WalkKernelFn = void (*)(const WalkArgs);
using BatchKernelFn = void (*)(const BatchArgs);

// ---------------------------------------------------------------------------
// Eq. 1 for a batch of permutations: one CTA per permutation.
// ---------------------------------------------------------------------------
template <typename FE, typename PE, int NT>
__global__ void __launch_bounds__(NT) cost_kernel(const FE* __restrict__ F, int ldF,
                                                 const PE* __restrict__ D, int n,
                                                 const int32_t* __restrict__ p, int count,
                                                 int64_t* __restrict__ out) {
  __shared__ int64_t red[32];
  for (int b = blockIdx.x; b < count; b += gridDim.x) {
    const int32_t* pb = p + (size_t)b * n;
    int64_t acc = 0;
    for (int c = threadIdx.x; c < n * n; c += NT) {
      const int i = c / n, j = c - (c / n) * n;
      acc += (int64_t)F[(size_t)i * ldF + j] * (int64_t)D[(size_t)pb[i] * n + pb[j]];
    }
    acc = block_sum<NT>(acc, red);
    if (threadIdx.x == 0) out[b] = acc;
  }
}

}  // namespace qapk
