// Walk kernels of the swap-neighbourhood QAP search (sm_103a).
//
// One CTA runs one search walk at a time and loops over walks (persistent
// form).  Per walk everything lives on chip:
//   shared memory   F (int16) and, for an asymmetric flow, its transpose;
//                   P = D[p][p] (int8) and, for asymmetric distances, its
//                   transpose; the tabu table (int32 per pair); the four
//                   O(1)-update vectors; the two recomputed delta rows;
//                   p and the best permutation.
//   registers       the delta of every pair the thread owns (thread t owns
//                   pairs t, t + NT, t + 2 NT, ... of the lexicographic
//                   pair order) and the packed (r << 8 | s) key of each.
//
// One iteration (Sections 4.1, 4.3):
//   scan    each thread filters its pairs (tabu / aspiration) and keeps the
//           lowest (delta, key); warp REDUX min, then one CTA-wide round
//           through shared memory gives every thread the chosen move;
//   apply   swap p[r], p[s]; swap rows and columns r, s of P (and P^T);
//           cost += delta; tabu stamp by the owner of (r, s);
//   update  pairs disjoint from {r, s}: O(1) update from the vectors
//             a_x = F[r][x]-F[s][x], b_x = P'[s][x]-P'[r][x],
//             c_x = F[x][r]-F[x][s], e_x = P'[x][s]-P'[x][r]
//           (delta += (a_u-a_v)(b_u-b_v) + (c_u-c_v)(e_u-e_v));
//           pairs touching r or s: Eq. 2 recomputed by 8-lane groups;
//           pair (r, s): negated.
#pragma once
#include <cstdint>
#include <climits>

#include "qap_philox.cuh"

namespace qapk {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kNoMove = 0xffffffffu;
constexpr uint32_t kNoPair = 0xffffu;  // packed-key slot without a pair
constexpr int kGroup = 8;  // lanes per recomputed pair
constexpr int kDescentCap = 1 << 20;  // 2opt moves when no cap is given

struct WalkArgs {
  int n, ldF, ldP;
  int symF, symD;
  const int16_t* F;   // n x ldF, row-major, padded
  const int16_t* Ft;  // transpose of F (== F when symF)
  const int8_t* D;    // n x n, row-major
  int walks;          // walks processed by this launch
  int walk_offset;    // index of this launch's first walk in the outputs
  uint32_t walk_base; // walk id of output row 0
  uint64_t seed;
  const int32_t* starts;  // (walk_offset + walks) x n, or null
  int descend, max_descent, iters;
  int tmin, tmax, period, aspiration;
  int32_t* best_p;
  int64_t* best_cost;
  int64_t* final_cost;
  int32_t* best_iter;
  int32_t* iters_done;
  int32_t* status;
  int32_t* descent_moves;
  uint64_t* hash;
  uint64_t* descent_hash;
};

// ---------------------------------------------------------------------------
// shared-memory layout (host and device agree through this function)
// ---------------------------------------------------------------------------
struct SmemLayout {
  int offF, offFt, offP, offPt, offTabu, offVec, offR, offPerm, offBest, offRedD, offRedK, offSum;
  int bytes;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

__host__ __device__ inline SmemLayout smem_layout(int n, int ldF, int ldP, int symF, int symD,
                                                  int dbytes) {
  SmemLayout L;
  const int T = n * (n - 1) / 2;
  int o = 0;
  L.offF = o;    o = align16(o + n * ldF * 2);
  L.offFt = o;   o = symF ? o : align16(o + n * ldF * 2);
  L.offP = o;    o = align16(o + n * ldP);
  L.offPt = o;   o = symD ? o : align16(o + n * ldP);
  L.offTabu = o; o = align16(o + T * 4);
  L.offVec = o;  o = align16(o + n * 16);
  L.offR = o;    o = align16(o + 2 * n * dbytes);
  L.offPerm = o; o = align16(o + n * 4);
  L.offBest = o; o = align16(o + n * 4);
  L.offRedD = o; o = align16(o + 32 * 8);
  L.offRedK = o; o = align16(o + 32 * 4);
  L.offSum = o;  o = align16(o + 32 * 8);
  L.bytes = o;
  return L;
}

template <typename DT> struct DeltaMax;
template <> struct DeltaMax<int32_t> { static constexpr int32_t v = INT_MAX; };
template <> struct DeltaMax<int64_t> { static constexpr int64_t v = LLONG_MAX; };

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
template <typename DT>
struct WalkSmem {
  int16_t* F;
  int16_t* Ft;
  int8_t* P;
  int8_t* Pt;
  int32_t* tabu;
  int4* vec;
  DT* R;
  int32_t* perm;
  int32_t* best;
  DT* redD;
  uint32_t* redK;
  int64_t* sum;
};

// Eq. 2 (with the diagonal term) for the pair {x, k}, by one thread.  The
// column terms of Eq. 2 read the transposed copies so every access is a row.
template <typename DT>
__device__ __forceinline__ DT delta_serial(const WalkSmem<DT>& S, int n, int ldF, int ldP,
                                           int sym, int x, int k) {
  const int16_t* Fx = S.F + x * ldF;
  const int16_t* Fk = S.F + k * ldF;
  const int8_t* Px = S.P + x * ldP;
  const int8_t* Pk = S.P + k * ldP;
  const int16_t* Ftx = S.Ft + x * ldF;
  const int16_t* Ftk = S.Ft + k * ldF;
  const int8_t* Ptx = S.Pt + x * ldP;
  const int8_t* Ptk = S.Pt + k * ldP;
  DT acc = 0;
  for (int j = 0; j < n; ++j) {
    if (j == x || j == k) continue;
    const int t1 = ((int)Fx[j] - (int)Fk[j]) * ((int)Pk[j] - (int)Px[j]);
    if (sym) {
      acc += (DT)(2 * t1);
    } else {
      const int t2 = ((int)Ftx[j] - (int)Ftk[j]) * ((int)Ptk[j] - (int)Ptx[j]);
      acc += (DT)t1 + (DT)t2;
    }
  }
  const int fixed = ((int)Fx[k] - (int)Fk[x]) * ((int)Pk[x] - (int)Px[k]);
  const int diag = ((int)Fx[x] - (int)Fk[k]) * ((int)Pk[k] - (int)Px[x]);
  return acc + (DT)fixed + (DT)diag;
}

// Apply move (r, s) to p and P (and P^T), then build the update vectors and
// the two recomputed delta rows.  Ends after a CTA barrier with S.vec and
// S.R valid for the owners' update.  `copy_best` also copies p' into best.
template <typename DT, int NT>
__device__ __forceinline__ void apply_move(const WalkSmem<DT>& S, int n, int ldF, int ldP,
                                           int symF, int symD, int r, int s, bool copy_best) {
  const int tid = threadIdx.x;
  const bool sym = symF && symD;
  if (tid == 0) {
    const int32_t t = S.perm[r];
    S.perm[r] = S.perm[s];
    S.perm[s] = t;
  }
  // P' = P with rows r, s and columns r, s exchanged.
  for (int j = tid; j < n; j += NT) {
    if (j != r && j != s) {
      int8_t* Pr = S.P + r * ldP;
      int8_t* Ps = S.P + s * ldP;
      int8_t t = Pr[j]; Pr[j] = Ps[j]; Ps[j] = t;
      int8_t* Pj = S.P + j * ldP;
      t = Pj[r]; Pj[r] = Pj[s]; Pj[s] = t;
      if (!symD) {
        int8_t* Qr = S.Pt + r * ldP;
        int8_t* Qs = S.Pt + s * ldP;
        t = Qr[j]; Qr[j] = Qs[j]; Qs[j] = t;
        int8_t* Qj = S.Pt + j * ldP;
        t = Qj[r]; Qj[r] = Qj[s]; Qj[s] = t;
      }
    } else if (j == r) {
      int8_t* Pr = S.P + r * ldP;
      int8_t* Ps = S.P + s * ldP;
      const int8_t rr = Pr[r], rs = Pr[s], sr = Ps[r], ss = Ps[s];
      Pr[r] = ss; Pr[s] = sr; Ps[r] = rs; Ps[s] = rr;
      if (!symD) {
        int8_t* Qr = S.Pt + r * ldP;
        int8_t* Qs = S.Pt + s * ldP;
        const int8_t qrr = Qr[r], qrs = Qr[s], qsr = Qs[r], qss = Qs[s];
        Qr[r] = qss; Qr[s] = qsr; Qs[r] = qrs; Qs[s] = qrr;
      }
    }
  }
  __syncthreads();

  if (copy_best)
    for (int x = tid; x < n; x += NT) S.best[x] = S.perm[x];

  // O(1)-update vectors from F and P'.
  {
    const int16_t* Fr = S.F + r * ldF;
    const int16_t* Fs = S.F + s * ldF;
    const int8_t* Pr = S.P + r * ldP;
    const int8_t* Ps = S.P + s * ldP;
    const int16_t* Ftr = S.Ft + r * ldF;
    const int16_t* Fts = S.Ft + s * ldF;
    const int8_t* Ptr = S.Pt + r * ldP;
    const int8_t* Pts = S.Pt + s * ldP;
    for (int x = tid; x < n; x += NT) {
      const int a = (int)Fr[x] - (int)Fs[x];
      const int b = (int)Ps[x] - (int)Pr[x];
      const int c = sym ? a : (int)Ftr[x] - (int)Fts[x];
      const int e = sym ? b : (int)Pts[x] - (int)Ptr[x];
      S.vec[x] = make_int4(a, b, c, e);
    }
  }

  // Eq. 2 recomputed for the pairs {r, k} (row 0 of R) and {s, k} (row 1),
  // k outside {r, s}; one 8-lane group per pair.
  {
    const int lane8 = tid & (kGroup - 1);
    const int group = tid / kGroup;
    constexpr int NG = NT / kGroup;
    const unsigned gmask = 0xffu << (threadIdx.x & 31 & ~(kGroup - 1));
    for (int q = group; q < 2 * n; q += NG) {
      const int xi = q >= n ? 1 : 0;
      const int k = q - xi * n;
      if (k == r || k == s) continue;
      const int x = xi ? s : r;
      const int16_t* Fx = S.F + x * ldF;
      const int16_t* Fk = S.F + k * ldF;
      const int8_t* Px = S.P + x * ldP;
      const int8_t* Pk = S.P + k * ldP;
      DT acc = 0;
      if (sym) {
        int part = 0;
        for (int j = lane8; j < n; j += kGroup) {
          const int t1 = ((int)Fx[j] - (int)Fk[j]) * ((int)Pk[j] - (int)Px[j]);
          part += (j == x || j == k) ? 0 : t1;
        }
        acc = (DT)2 * (DT)part;
      } else {
        const int16_t* Ftx = S.Ft + x * ldF;
        const int16_t* Ftk = S.Ft + k * ldF;
        const int8_t* Ptx = S.Pt + x * ldP;
        const int8_t* Ptk = S.Pt + k * ldP;
        for (int j = lane8; j < n; j += kGroup) {
          const int t1 = ((int)Fx[j] - (int)Fk[j]) * ((int)Pk[j] - (int)Px[j]);
          const int t2 = ((int)Ftx[j] - (int)Ftk[j]) * ((int)Ptk[j] - (int)Ptx[j]);
          acc += (j == x || j == k) ? (DT)0 : (DT)t1 + (DT)t2;
        }
      }
#pragma unroll
      for (int o = kGroup / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(gmask, acc, o);
      if (lane8 == 0) {
        const int fixed = ((int)Fx[k] - (int)Fk[x]) * ((int)Pk[x] - (int)Px[k]);
        const int diag = ((int)Fx[x] - (int)Fk[k]) * ((int)Pk[k] - (int)Px[x]);
        S.R[xi * n + k] = acc + (DT)fixed + (DT)diag;
      }
    }
  }
  __syncthreads();
}

// New delta of an owned pair after move (r, s) (vectors and rows ready).
template <typename DT>
__device__ __forceinline__ DT updated_delta(const WalkSmem<DT>& S, int n, DT d, uint32_t key,
                                            uint32_t rs, int r, int s) {
  const int u = (int)(key >> 8), v = (int)(key & 0xffu);
  if (key == rs) return -d;
  if (u == r || v == r) return S.R[u == r ? v : u];
  if (u == s || v == s) return S.R[n + (u == s ? v : u)];
  const int4 A = S.vec[u], B = S.vec[v];
  return d + (DT)((A.x - B.x) * (A.y - B.y) + (A.z - B.z) * (A.w - B.w));
}

// ---------------------------------------------------------------------------
// the walk kernel
// ---------------------------------------------------------------------------
constexpr int min_blocks(int nt) { return nt <= 128 ? 4 : nt <= 256 ? 2 : 1; }

template <typename DT, int NT, int MAXPT>
__global__ void __launch_bounds__(NT, min_blocks(NT)) walk_kernel(const WalkArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, ldF = a.ldF, ldP = a.ldP, tid = threadIdx.x;
  const int T = n * (n - 1) / 2;
  const bool sym = a.symF && a.symD;
  const SmemLayout L = smem_layout(n, ldF, ldP, a.symF, a.symD, (int)sizeof(DT));
  WalkSmem<DT> S;
  S.F = reinterpret_cast<int16_t*>(smem + L.offF);
  S.Ft = a.symF ? S.F : reinterpret_cast<int16_t*>(smem + L.offFt);
  S.P = reinterpret_cast<int8_t*>(smem + L.offP);
  S.Pt = a.symD ? S.P : reinterpret_cast<int8_t*>(smem + L.offPt);
  S.tabu = reinterpret_cast<int32_t*>(smem + L.offTabu);
  S.vec = reinterpret_cast<int4*>(smem + L.offVec);
  S.R = reinterpret_cast<DT*>(smem + L.offR);
  S.perm = reinterpret_cast<int32_t*>(smem + L.offPerm);
  S.best = reinterpret_cast<int32_t*>(smem + L.offBest);
  S.redD = reinterpret_cast<DT*>(smem + L.offRedD);
  S.redK = reinterpret_cast<uint32_t*>(smem + L.offRedK);
  S.sum = reinterpret_cast<int64_t*>(smem + L.offSum);

  // Owned pairs: linear index tid + i*NT in lexicographic (u, v) order; the
  // 16-bit keys (u << 8 | v) of two slots share one register.
  static_assert(MAXPT % 2 == 0, "keys are packed in pairs");
  uint32_t kp[MAXPT / 2];
  {
    int u = 0, rowStart = 0;
#pragma unroll
    for (int i = 0; i < MAXPT; ++i) {
      const int q = tid + i * NT;
      uint32_t k16 = kNoPair;
      if (q < T) {
        while (q >= rowStart + (n - 1 - u)) {
          rowStart += n - 1 - u;
          ++u;
        }
        k16 = ((uint32_t)u << 8) | (uint32_t)(u + 1 + (q - rowStart));
      }
      if (i & 1) kp[i / 2] |= k16 << 16;
      else kp[i / 2] = k16;
    }
  }
#define QAP_KEY(i) ((kp[(i) / 2] >> (16 * ((i) & 1))) & 0xffffu)

  // F (and F^T) once per CTA: rows are whole 16-byte vectors.
  {
    const int nvec = n * ldF * 2 / 16;
    const int4* gF = reinterpret_cast<const int4*>(a.F);
    int4* sF = reinterpret_cast<int4*>(S.F);
    for (int i = tid; i < nvec; i += NT) sF[i] = gF[i];
    if (!a.symF) {
      const int4* gFt = reinterpret_cast<const int4*>(a.Ft);
      int4* sFt = reinterpret_cast<int4*>(S.Ft);
      for (int i = tid; i < nvec; i += NT) sFt[i] = gFt[i];
    }
  }

  for (int w = blockIdx.x; w < a.walks; w += gridDim.x) {
    const int wi = a.walk_offset + w;
    const uint32_t wid = a.walk_base + (uint32_t)wi;

    // Start permutation: given, or Fisher-Yates on stream 0.
    if (a.starts) {
      for (int x = tid; x < n; x += NT) S.perm[x] = a.starts[(size_t)wi * n + x];
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
    for (int c = tid; c < n * n; c += NT) {
      const int i = c / n, j = c - (c / n) * n;
      const int8_t v = a.D[(size_t)S.perm[i] * n + S.perm[j]];
      S.P[i * ldP + j] = v;
      if (!a.symD) S.Pt[j * ldP + i] = v;
    }
    for (int x = tid; x < n; x += NT) S.best[x] = S.perm[x];
    __syncthreads();

    // Eq. 1.
    int64_t c0 = 0;
    for (int c = tid; c < n * n; c += NT) {
      const int i = c / n, j = c - (c / n) * n;
      c0 += (int64_t)S.F[i * ldF + j] * (int64_t)S.P[i * ldP + j];
    }
    c0 = block_sum<NT>(c0, S.sum);

    // Initial deltas of the owned pairs (Eq. 2, O(n) each) and tabu table.
    DT dl[MAXPT];
#pragma unroll
    for (int i = 0; i < MAXPT; ++i) {
      dl[i] = 0;
      if (QAP_KEY(i) != kNoPair) {
        dl[i] = delta_serial<DT>(S, n, ldF, ldP, sym, (int)(QAP_KEY(i) >> 8), (int)(QAP_KEY(i) & 0xffu));
        S.tabu[tid + i * NT] = 0;
      }
    }

    DT cur = (DT)c0;
    uint64_t h = 14695981039346656037ull, dh = h;
    int dmoves = 0;

    // ---- 2opt descent (Section 4.1): best move while it improves.
    if (a.descend) {
      // A descent strictly lowers the cost at every move, so it ends; the
      // cap only bounds the kernel's run time on any input.
      const int cap = a.max_descent >= 0 ? a.max_descent : kDescentCap;
      for (;;) {
        if (dmoves >= cap) break;
        DT bd = DeltaMax<DT>::v;
        uint32_t bk = kNoMove;
#pragma unroll
        for (int i = 0; i < MAXPT; ++i)
          if (QAP_KEY(i) != kNoPair && dl[i] < bd) {
            bd = dl[i];
            bk = QAP_KEY(i);
          }
        block_argmin<DT, NT>(bd, bk, S.redD, S.redK);
        if (bk == kNoMove || bd >= 0) break;
        const int r = (int)(bk >> 8), s = (int)(bk & 0xffu);
        cur += bd;
        ++dmoves;
        dh = fnv_step(dh, r, s);
        apply_move<DT, NT>(S, n, ldF, ldP, a.symF, a.symD, r, s, false);
#pragma unroll
        for (int i = 0; i < MAXPT; ++i)
          if (QAP_KEY(i) != kNoPair) dl[i] = updated_delta<DT>(S, n, dl[i], QAP_KEY(i), bk, r, s);
      }
      __syncthreads();
      for (int x = tid; x < n; x += NT) S.best[x] = S.perm[x];
    }

    // ---- tabu search (Sections 4.3, 4.4).
    DT best = cur;
    int best_iter = 0, status = 0, done = 0;
    for (int it = 1; it <= a.iters; ++it) {
      DT bd = DeltaMax<DT>::v;
      uint32_t bk = kNoMove;
#pragma unroll
      for (int i = 0; i < MAXPT; ++i) {
        if (QAP_KEY(i) == kNoPair) continue;
        const DT d = dl[i];
        const bool adm = S.tabu[tid + i * NT] <= it || (a.aspiration && cur + d < best);
        if (adm && d < bd) {
          bd = d;
          bk = QAP_KEY(i);
        }
      }
      block_argmin<DT, NT>(bd, bk, S.redD, S.redK);
      if (bk == kNoMove) {
        status = 1;
        break;
      }
      const int r = (int)(bk >> 8), s = (int)(bk & 0xffu);
      cur += bd;
      done = it;
      h = fnv_step(h, r, s);
      const bool improved = cur < best;
      if (improved) {
        best = cur;
        best_iter = it;
      }
#pragma unroll
      for (int i = 0; i < MAXPT; ++i) {
        if (QAP_KEY(i) == bk) {
          const uint32_t k = a.period > 0 ? (uint32_t)((it - 1) / a.period) : (uint32_t)(it - 1);
          const uint32_t x = walk_draw(a.seed, wid, 1u, k);
          S.tabu[tid + i * NT] = it + a.tmin + (int)below(x, (uint32_t)(a.tmax - a.tmin + 1));
        }
      }
      apply_move<DT, NT>(S, n, ldF, ldP, a.symF, a.symD, r, s, improved);
#pragma unroll
      for (int i = 0; i < MAXPT; ++i)
        if (QAP_KEY(i) != kNoPair) dl[i] = updated_delta<DT>(S, n, dl[i], QAP_KEY(i), bk, r, s);
    }
    __syncthreads();

    // ---- outputs
    if (a.best_p)
      for (int x = tid; x < n; x += NT) a.best_p[(size_t)wi * n + x] = S.best[x];
    if (tid == 0) {
      a.best_cost[wi] = (int64_t)best;
      if (a.final_cost) a.final_cost[wi] = (int64_t)cur;
      if (a.best_iter) a.best_iter[wi] = best_iter;
      if (a.iters_done) a.iters_done[wi] = done;
      if (a.status) a.status[wi] = status;
      if (a.descent_moves) a.descent_moves[wi] = dmoves;
      if (a.hash) a.hash[wi] = h;
      if (a.descent_hash) a.descent_hash[wi] = dh;
    }
    __syncthreads();
  }
#undef QAP_KEY
}

using WalkKernelFn = void (*)(const WalkArgs);

// ---------------------------------------------------------------------------
// Eq. 1 for a batch of permutations: one CTA per permutation.
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(NT) cost_kernel(const int16_t* __restrict__ F, int ldF,
                                                 const int8_t* __restrict__ D, int n,
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
