// Probe of the phase-X contraction of one tabu iteration on two units: the
// integer dot-product units (dp4a, as the walk kernel does it) and the
// tensor cores (mma.sync m16n8k16, f16 inputs, f32 accumulation).
//
// Per iteration, for a move (r, s) of an n x n instance with int8 values:
//   Ar[k] = F[r].Q[k] + F^T[r].Q^T[k]     As[k] = F[s].Q[k] + F^T[s].Q^T[k]
//   Br[k] = F[k].Q[s] + F^T[k].Q^T[s]     Bs[k] = F[k].Q[r] + F^T[k].Q^T[r]
// for every k: matrix-vector products of length 2n (the dot products of
// Eq. 2 for the pairs touching r and s).  f16 holds the int8 values exactly
// and f32 the sums (below 2 n 127^2 < 2^24 for n <= 128), so both forms are
// exact and give the same numbers.  One CTA of 256 threads per instance
// copy; the probe times `iters` iterations of each form and prints
//   n=<n> dp4a_us=<per iteration> mma_us=<per iteration> equal=<0|1>
// Built and run by tests/test_gpu_mma_probe.py; not part of the library.
//
// The tensor-core form multiplies the n x 4n matrix whose row k is
// [Q[k] | Q^T[k] | F[k] | F^T[k]] (f16, laid out once) by a 4n x 8 matrix
// built per iteration: column 0 = [F[r] | F^T[r] | 0 | 0], column 1 the same
// for s, column 2 = [0 | 0 | Q[s] | Q^T[s]], column 3 the same for r,
// columns 4-7 zero.  Output columns 0-3 are Ar, As, Br, Bs.  The move
// changes only the small matrix, so this is the form with the least
// per-iteration work on the tensor cores; half of every B operand and half
// of the output tile are zeros by construction (the products have 4
// columns, the instruction 8).
#include <cuda_fp16.h>

#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

namespace {

constexpr int NT = 256;
constexpr int NMAX = 128;
constexpr int LD = NMAX;            // int8 row stride (elements)
constexpr int LDA = 4 * NMAX + 8;   // f16 row stride of the big operand (padding spreads banks)

struct Smem {
  int8_t F[NMAX * LD], Ft[NMAX * LD], Q[NMAX * LD], Qt[NMAX * LD];
  __half A[NMAX * LDA];   // row k: [Q[k] | Q^T[k] | F[k] | F^T[k]], each part npad wide
  __half Bt[8 * LDA];     // the small operand, transposed: row c = column c of B
};

__device__ __forceinline__ void move_of(int it, int n, int* r, int* s) {
  const int a = it % n, b = (it * 7 + 3) % n;
  *r = a;
  *s = b == a ? (a + 1) % n : b;
}

__device__ void load(Smem& S, const int8_t* F, const int8_t* Q, int n, int npad) {
  for (int e = threadIdx.x; e < NMAX * LD; e += NT) {
    const int i = e / LD, j = e % LD;
    const bool in = i < n && j < n;
    S.F[e] = in ? F[i * n + j] : 0;
    S.Ft[e] = in ? F[j * n + i] : 0;
    S.Q[e] = in ? Q[i * n + j] : 0;
    S.Qt[e] = in ? Q[j * n + i] : 0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NMAX * 4 * npad; e += NT) {
    const int k = e / (4 * npad), j = e % (4 * npad), part = j / npad, c = j % npad;
    const int8_t* m = part == 0 ? S.Q : part == 1 ? S.Qt : part == 2 ? S.F : S.Ft;
    S.A[k * LDA + j] = __int2half_rn(m[k * LD + c]);
  }
  for (int e = threadIdx.x; e < 8 * LDA; e += NT) S.Bt[e] = __float2half(0.f);
  __syncthreads();
}

// dp4a, organised as the walk kernel's phase X: one index k per group of G
// lanes (the widest power of two up to 8 that still gives every k its own
// group), the lanes of a group splitting the rows' 16-byte chunks; the k-row
// chunks serve all four products, which accumulate side by side; a shuffle
// reduction over the group finishes them.
__global__ void __launch_bounds__(NT) dp4a_kernel(const int8_t* F, const int8_t* Q, int n,
                                                  int iters, unsigned* out) {
  extern __shared__ __align__(16) unsigned char raw[];
  Smem& S = *reinterpret_cast<Smem*>(raw);
  load(S, F, Q, n, (n + 15) / 16 * 16);
  const int nc = (n + 15) / 16;
  int G = 8;
  while (G > 1 && (NT / G < n || G > nc)) G >>= 1;
  const int lg = threadIdx.x & (G - 1), grp = threadIdx.x / G;
  unsigned acc = 0;
  for (int it = 0; it < iters; ++it) {
    int r, s;
    move_of(it, n, &r, &s);
    const int4* Fr = reinterpret_cast<const int4*>(S.F + r * LD);
    const int4* Fs = reinterpret_cast<const int4*>(S.F + s * LD);
    const int4* Ftr = reinterpret_cast<const int4*>(S.Ft + r * LD);
    const int4* Fts = reinterpret_cast<const int4*>(S.Ft + s * LD);
    const int4* Qr = reinterpret_cast<const int4*>(S.Q + r * LD);
    const int4* Qs = reinterpret_cast<const int4*>(S.Q + s * LD);
    const int4* Qtr = reinterpret_cast<const int4*>(S.Qt + r * LD);
    const int4* Qts = reinterpret_cast<const int4*>(S.Qt + s * LD);
    for (int base = 0; base < n; base += NT / G) {
      const int k = min(base + grp, n - 1);
      const int4* Fk = reinterpret_cast<const int4*>(S.F + k * LD);
      const int4* Ftk = reinterpret_cast<const int4*>(S.Ft + k * LD);
      const int4* Qk = reinterpret_cast<const int4*>(S.Q + k * LD);
      const int4* Qtk = reinterpret_cast<const int4*>(S.Qt + k * LD);
      int Ar = 0, As = 0, Br = 0, Bs = 0;
      auto dot = [](int4 a, int4 b, int c) {
        c = __dp4a(a.x, b.x, c);
        c = __dp4a(a.y, b.y, c);
        c = __dp4a(a.z, b.z, c);
        return __dp4a(a.w, b.w, c);
      };
      for (int c = lg; c < nc; c += G) {
        const int4 fk = Fk[c], ftk = Ftk[c], qk = Qk[c], qtk = Qtk[c];
        Ar = dot(Fr[c], qk, dot(Ftr[c], qtk, Ar));
        As = dot(Fs[c], qk, dot(Fts[c], qtk, As));
        Br = dot(fk, Qs[c], dot(ftk, Qts[c], Br));
        Bs = dot(fk, Qr[c], dot(ftk, Qtr[c], Bs));
      }
      for (int o = 1; o < G; o <<= 1) {
        Ar += __shfl_xor_sync(0xffffffffu, Ar, o);
        As += __shfl_xor_sync(0xffffffffu, As, o);
        Br += __shfl_xor_sync(0xffffffffu, Br, o);
        Bs += __shfl_xor_sync(0xffffffffu, Bs, o);
      }
      if (lg == 0 && base + grp < n)
        acc += (unsigned)Ar + 3u * (unsigned)As + 5u * (unsigned)Br + 7u * (unsigned)Bs;
    }
    __syncthreads();
  }
  out[blockIdx.x * NT + threadIdx.x] = acc;
}

__global__ void __launch_bounds__(NT) mma_kernel(const int8_t* F, const int8_t* Q, int n,
                                                 int iters, unsigned* out) {
  extern __shared__ __align__(16) unsigned char raw[];
  Smem& S = *reinterpret_cast<Smem*>(raw);
  const int npad = (n + 15) / 16 * 16;
  load(S, F, Q, n, npad);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const int K = 4 * npad, ksteps = K / 16, mtiles = (n + 15) / 16;
  unsigned acc = 0;
  for (int it = 0; it < iters; ++it) {
    int r, s;
    move_of(it, n, &r, &s);
    // columns 0-3 of the small operand for this move
    for (int e = threadIdx.x; e < 4 * K; e += NT) {
      const int c = e / K, j = e % K, part = j / npad, x = j % npad;
      const int row = c == 0 ? r : c == 1 ? s : c == 2 ? s : r;
      int8_t v = 0;
      if (c < 2 && part < 2) v = (part == 0 ? S.F : S.Ft)[row * LD + x];
      if (c >= 2 && part >= 2) v = (part == 2 ? S.Q : S.Qt)[row * LD + x];
      S.Bt[c * LDA + j] = __int2half_rn(v);
    }
    __syncthreads();
    for (int mt = warp; mt < mtiles; mt += NT / 32) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      const __half* A0 = S.A + (mt * 16 + g) * LDA + 2 * tq;
      const __half* A1 = A0 + 8 * LDA;
      const __half* B0 = S.Bt + g * LDA + 2 * tq;
      for (int ks = 0; ks < ksteps; ++ks) {
        const int j0 = ks * 16;
        const unsigned a0 = *reinterpret_cast<const unsigned*>(A0 + j0);
        const unsigned a1 = *reinterpret_cast<const unsigned*>(A1 + j0);
        const unsigned a2 = *reinterpret_cast<const unsigned*>(A0 + j0 + 8);
        const unsigned a3 = *reinterpret_cast<const unsigned*>(A1 + j0 + 8);
        const unsigned b0 = *reinterpret_cast<const unsigned*>(B0 + j0);
        const unsigned b1 = *reinterpret_cast<const unsigned*>(B0 + j0 + 8);
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
            "{%8,%9}, {%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
      }
      // c0, c1: row mt*16 + g, columns 2 tq and 2 tq + 1; c2, c3: row + 8
      for (int h = 0; h < 2; ++h) {
        const int k = mt * 16 + g + 8 * h;
        for (int e = 0; e < 2; ++e) {
          const int q = 2 * tq + e;
          if (k < n && q < 4) acc += (unsigned)(int)c[2 * h + e] * (unsigned)(2 * q + 1);
        }
      }
    }
    __syncthreads();
  }
  out[blockIdx.x * NT + threadIdx.x] = acc;
}

}  // namespace

int main(int argc, char** argv) {
  const int n = argc > 1 ? atoi(argv[1]) : 100;
  const int iters = argc > 2 ? atoi(argv[2]) : 2000;
  const int ctas = argc > 3 ? atoi(argv[3]) : 152;
  if (n < 2 || n > NMAX || iters < 1 || ctas < 1) return 2;
  std::vector<int8_t> F(n * n), Q(n * n);
  unsigned x = 12345;
  for (int i = 0; i < n * n; ++i) {
    x = x * 1103515245u + 12345u;
    F[i] = (int8_t)((x >> 16) % 100);
    x = x * 1103515245u + 12345u;
    Q[i] = (int8_t)((x >> 16) % 100);
  }
  int8_t *dF = nullptr, *dQ = nullptr;
  unsigned *o1 = nullptr, *o2 = nullptr;
  cudaMalloc(&dF, n * n);
  cudaMalloc(&dQ, n * n);
  cudaMalloc(&o1, ctas * NT * sizeof(unsigned));
  cudaMalloc(&o2, ctas * NT * sizeof(unsigned));
  cudaMemcpy(dF, F.data(), n * n, cudaMemcpyHostToDevice);
  cudaMemcpy(dQ, Q.data(), n * n, cudaMemcpyHostToDevice);
  const int smem = (int)sizeof(Smem);
  cudaFuncSetAttribute(dp4a_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float t1 = 0, t2 = 0;
  for (int rep = 0; rep < 2; ++rep) {  // warm-up, then timed
    cudaEventRecord(a);
    dp4a_kernel<<<ctas, NT, smem>>>(dF, dQ, n, iters, o1);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&t1, a, b);
    cudaEventRecord(a);
    mma_kernel<<<ctas, NT, smem>>>(dF, dQ, n, iters, o2);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&t2, a, b);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    printf("cuda error: %s\n", cudaGetErrorString(e));
    return 1;
  }
  // per CTA, the sums over all threads (mod 2^32) must agree: the two forms
  // split the work over threads differently
  std::vector<unsigned> h1(ctas * NT), h2(ctas * NT);
  cudaMemcpy(h1.data(), o1, h1.size() * sizeof(unsigned), cudaMemcpyDeviceToHost);
  cudaMemcpy(h2.data(), o2, h2.size() * sizeof(unsigned), cudaMemcpyDeviceToHost);
  bool equal = true;
  for (int c = 0; c < ctas; ++c) {
    unsigned s1 = 0, s2 = 0;
    for (int t = 0; t < NT; ++t) {
      s1 += h1[c * NT + t];
      s2 += h2[c * NT + t];
    }
    equal &= s1 == s2;
  }
  printf("n=%d dp4a_us=%.4f mma_us=%.4f equal=%d\n", n, 1e3 * t1 / iters, 1e3 * t2 / iters,
         equal ? 1 : 0);
  cudaFree(dF);
  cudaFree(dQ);
  cudaFree(o1);
  cudaFree(o2);
  return equal ? 0 : 1;
}
