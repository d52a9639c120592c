// Shared-memory mixed-radix FFT core, in place, register-blocked stages.
//
// Forward transforms run decimation-in-frequency stages: natural-order input,
// output left in the mixed-radix digit-reversed order of the plan (frequency k
// sits at position fft_pos(k)).  Inverse transforms run the exact stage
// inverses in reverse order: digit-reversed input, natural-order output,
// unnormalised (sum_k X[k] e^{+2 pi i n k / L}).  A forward + pointwise +
// inverse sequence therefore never needs a reordering pass.
//
// One stage of block length Lb = R * M maps, for every n1 < M,
//   x[n1 + M n2] -> y[k2] = W_Lb^{n1 k2} sum_n2 x[n1 + M n2] W_R^{n2 k2}
// stored back at n1 + M k2.  Each thread keeps the R points of a butterfly in
// registers, so a stage is one shared-memory round trip; radices up to 16
// (composite ones as two register levels) keep lengths such as 2160 = 16 15 9
// to three stages.  Stage twiddles W_Lb^{n1 k} (k = 1 .. R-1, n1 < Lb / R)
// come from per-stage tables, each value rounded once from FP64.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "mm_internal.h"

namespace mm {

template <typename C> struct cplx_traits;
template <> struct cplx_traits<float2> { typedef float real; };
template <> struct cplx_traits<double2> { typedef double real; };

template <typename C> __device__ __forceinline__ C cmake(typename cplx_traits<C>::real x,
                                                         typename cplx_traits<C>::real y) {
  C c; c.x = x; c.y = y; return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cmulconj(C a, C b) {  // a * conj(b)
  return cmake<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ C cscale(C a, typename cplx_traits<C>::real s) {
  return cmake<C>(a.x * s, a.y * s);
}
// multiply by i*s (s = +-1)
template <typename C> __device__ __forceinline__ C cmul_is(C a, int s) {
  return s > 0 ? cmake<C>(-a.y, a.x) : cmake<C>(a.y, -a.x);
}

// cos / sin of 2 pi j / 720 for j < 720 (720 is a multiple of every radix),
// one copy per translation unit, filled by upload_roots();
// W_R^j = (c[j * 720/R], s[j * 720/R]).
constexpr int kRootN = 720;
static __constant__ float c_root_f[2][kRootN];
static __constant__ double c_root_d[2][kRootN];

static inline cudaError_t upload_roots() {
  static float rf[2][kRootN];
  static double rd[2][kRootN];
  for (int j = 0; j < kRootN; ++j) {
    const double a = 2.0 * 3.14159265358979323846 * (double)j / (double)kRootN;
    rd[0][j] = cos(a);
    rd[1][j] = sin(a);
    rf[0][j] = (float)rd[0][j];
    rf[1][j] = (float)rd[1][j];
  }
  cudaError_t e = cudaMemcpyToSymbol(c_root_f, rf, sizeof(rf));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_root_d, rd, sizeof(rd));
  return e;
}

template <typename C> __device__ __forceinline__ C root(int j);  // exp(+2 pi i j / kRootN)
template <> __device__ __forceinline__ float2 root<float2>(int j) {
  return make_float2(c_root_f[0][j], c_root_f[1][j]);
}
template <> __device__ __forceinline__ double2 root<double2>(int j) {
  return make_double2(c_root_d[0][j], c_root_d[1][j]);
}

// Small DFTs y[k] = sum_n x[n] exp(s 2 pi i n k / R) in registers.
template <int R, typename C> struct Dft;

template <typename C> struct Dft<2, C> {
  static __device__ __forceinline__ void run(C* x, int) {
    C a = x[0], b = x[1];
    x[0] = cadd(a, b); x[1] = csub(a, b);
  }
};
template <typename C> struct Dft<3, C> {
  static __device__ __forceinline__ void run(C* x, int s) {
    typedef typename cplx_traits<C>::real R;
    const R h = (R)0.86602540378443864676;  // sqrt(3)/2
    C t = cadd(x[1], x[2]);
    C m = csub(x[0], cscale(t, (R)0.5));
    C id = cmul_is(cscale(csub(x[1], x[2]), h), s);
    x[0] = cadd(x[0], t);
    x[1] = cadd(m, id);
    x[2] = csub(m, id);
  }
};
template <typename C> struct Dft<4, C> {
  static __device__ __forceinline__ void run(C* x, int s) {
    C a = cadd(x[0], x[2]), b = csub(x[0], x[2]);
    C c = cadd(x[1], x[3]), d = cmul_is(csub(x[1], x[3]), s);
    x[0] = cadd(a, c); x[2] = csub(a, c);
    x[1] = cadd(b, d); x[3] = csub(b, d);
  }
};
template <typename C> struct Dft<5, C> {
  static __device__ __forceinline__ void run(C* x, int s) {
    typedef typename cplx_traits<C>::real R;
    const R c1 = (R)0.30901699437494742410;   // cos(2 pi / 5)
    const R c2 = (R)-0.80901699437494742410;  // cos(4 pi / 5)
    const R s1 = (R)0.95105651629515357212;   // sin(2 pi / 5)
    const R s2 = (R)0.58778525229247312917;   // sin(4 pi / 5)
    C t1 = cadd(x[1], x[4]), t2 = cadd(x[2], x[3]);
    C d1 = csub(x[1], x[4]), d2 = csub(x[2], x[3]);
    C a1 = cadd(x[0], cadd(cscale(t1, c1), cscale(t2, c2)));
    C a2 = cadd(x[0], cadd(cscale(t1, c2), cscale(t2, c1)));
    C b1 = cmul_is(cadd(cscale(d1, s1), cscale(d2, s2)), s);
    C b2 = cmul_is(csub(cscale(d1, s2), cscale(d2, s1)), s);
    x[0] = cadd(x[0], cadd(t1, t2));
    x[1] = cadd(a1, b1); x[4] = csub(a1, b1);
    x[2] = cadd(a2, b2); x[3] = csub(a2, b2);
  }
};

// Composite R = A * B: n = B n1 + n2, k = k1 + A k2,
//   y[k1 + A k2] = sum_n2 W_B^{n2 k2} W_R^{n2 k1} sum_n1 x[B n1 + n2] W_A^{n1 k1}
template <int A, int B, typename C> struct DftComp {
  static __device__ __forceinline__ void run(C* x, int s) {
    constexpr int R = A * B;
    C t[B][A];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) {
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) t[n2][n1] = x[B * n1 + n2];
      Dft<A, C>::run(t[n2], s);
#pragma unroll
      for (int k1 = 1; k1 < A; ++k1) {
        if (n2 == 0) continue;
        const int j = (n2 * k1) % R * (kRootN / R);
        C w = root<C>(j);
        if (s < 0) w.y = -w.y;
        t[n2][k1] = cmul(t[n2][k1], w);
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      C u[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) u[n2] = t[n2][k1];
      Dft<B, C>::run(u, s);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) x[k1 + A * k2] = u[k2];
    }
  }
};
// Coprime R = A * B (Good-Thomas prime-factor mapping): with
// n = (B n1 + A n2) mod R and k = the k' < R with k' = k1 (mod A), k' = k2 (mod B),
//   y[k] = sum_n2 W_B^{n2 k2} sum_n1 x[(B n1 + A n2) mod R] W_A^{n1 k1},
// with no twiddle factors between the two levels.
__host__ __device__ constexpr int inv_mod(int a, int m) {
  int r = 1;
  while ((a * r) % m != 1) ++r;
  return r;
}
template <int A, int B, typename C> struct DftPfa {
  static __device__ __forceinline__ void run(C* x, int s) {
    constexpr int R = A * B;
    constexpr int eA = B * inv_mod(B % A, A);  // = 1 (mod A), = 0 (mod B)
    constexpr int eB = A * inv_mod(A % B, B);  // = 0 (mod A), = 1 (mod B)
    C t[B][A];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) {
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) t[n2][n1] = x[(B * n1 + A * n2) % R];
      Dft<A, C>::run(t[n2], s);
    }
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      C u[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) u[n2] = t[n2][k1];
      Dft<B, C>::run(u, s);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) x[(k1 * eA + k2 * eB) % R] = u[k2];
    }
  }
};
template <typename C> struct Dft<6, C> : DftPfa<2, 3, C> {};
template <typename C> struct Dft<8, C> : DftComp<2, 4, C> {};
template <typename C> struct Dft<9, C> : DftComp<3, 3, C> {};
template <typename C> struct Dft<10, C> : DftPfa<2, 5, C> {};
template <typename C> struct Dft<12, C> : DftPfa<4, 3, C> {};
template <typename C> struct Dft<15, C> : DftPfa<3, 5, C> {};
template <typename C> struct Dft<16, C> : DftComp<4, 4, C> {};


// Stage twiddles w[k] = W_Lb^{n1 k}, k = 1..R-1: entry (k - 1) M + n1 of the
// stage table, so the lanes of a warp (consecutive n1) read consecutive words.
template <int R, typename C>
__device__ __forceinline__ void stage_twiddles(const C* __restrict__ col, int M, C* w) {
#pragma unroll
  for (int k = 1; k < R; ++k) w[k] = col[(k - 1) * M];
}

// PRUNE (first forward stage only, Lb = L): inputs at or beyond `nvalid` are
// zero padding, taken as zero without being read (or ever written).
template <int R, bool INV, typename C, bool PRUNE = false>
__device__ __forceinline__ void fft_stage(C* buf, int ldl, int nlines, int L, int Lb, unsigned mpl,
                                          unsigned mM, const C* __restrict__ stw, int tid, int nthr,
                                          int nvalid = 0) {
  const int M = Lb / R;
  const int per_line = L / R;
  const int nb = nlines * per_line;
  for (int b = tid; b < nb; b += nthr) {
    const int line = mpl ? (int)__umulhi((unsigned)b, mpl) : b;
    const int rem = b - line * per_line;
    const int blk = mM ? (int)__umulhi((unsigned)rem, mM) : rem;
    const int n1 = rem - blk * M;
    C* base = buf + (line * ldl + blk * Lb + n1);  // shared memory: 32-bit offsets
    C v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = (!PRUNE || n1 + k * M < nvalid) ? base[k * M] : cmake<C>(0, 0);
    if (!INV) {
      Dft<R, C>::run(v, -1);
      if (n1) {
        C w[R];
        stage_twiddles<R, C>(stw + n1, M, w);
#pragma unroll
        for (int k = 1; k < R; ++k) v[k] = cmul(v[k], w[k]);
      }
    } else {
      if (n1) {
        C w[R];
        stage_twiddles<R, C>(stw + n1, M, w);
#pragma unroll
        for (int k = 1; k < R; ++k) v[k] = cmulconj(v[k], w[k]);
      }
      Dft<R, C>::run(v, +1);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) base[k * M] = v[k];
  }
}

// Decimation-in-frequency stage with the inverse sign: natural-order input,
// digit-reversed output of sum_k X[k] e^{+2 pi i n k / L}.
template <int R, typename C>
__device__ __forceinline__ void fft_stage_dif_inv(C* buf, int ldl, int nlines, int L, int Lb, unsigned mpl,
                                                  unsigned mM, const C* __restrict__ stw, int tid, int nthr) {
  const int M = Lb / R;
  const int per_line = L / R;
  const int nb = nlines * per_line;
  for (int b = tid; b < nb; b += nthr) {
    const int line = mpl ? (int)__umulhi((unsigned)b, mpl) : b;
    const int rem = b - line * per_line;
    const int blk = mM ? (int)__umulhi((unsigned)rem, mM) : rem;
    const int n1 = rem - blk * M;
    C* base = buf + (line * ldl + blk * Lb + n1);
    C v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = base[k * M];
    Dft<R, C>::run(v, +1);
    if (n1) {
      C w[R];
      stage_twiddles<R, C>(stw + n1, M, w);
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmulconj(v[k], w[k]);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) base[k * M] = v[k];
  }
}

// Stage orders of fft_smem.
enum FftMode { kFwdDif = 0, kInvDit = 1, kInvDif = 2 };

// Radix sets (radix_bit, kRadixSetA in mm_internal.h): a kernel instantiated
// for a set carries the stage code of those radices only; compact code for the
// radices a plan actually uses measured several per cent faster than the
// kernel with every radix compiled in.
inline unsigned plan_radix_set(const FftPlanDev& P) {
  unsigned s = 0;
  for (int i = 0; i < P.nstages; ++i) s |= radix_bit(P.radix[i]);
  return s;
}

// Runs all stages of one transform on `nlines` lines of buf (line stride ldl),
// using the threads [tid0, tid0 + nthr) of the block.  The caller syncs before.
//   kFwdDif: forward, natural in, digit-reversed out
//   kInvDit: inverse, digit-reversed in, natural out
//   kInvDif: inverse, natural in, digit-reversed out
// stw: the stage twiddle tables of the plan (stage s at P.stw_off[s]).
// nvalid (kFwdDif): 0 < nvalid < L means entries [nvalid, L) of every line
// are zero padding that the caller need not write.
template <int MODE, typename C, unsigned RSET = kAllRadices>
__device__ __forceinline__ void fft_smem(C* buf, int ldl, int nlines, const FftPlanDev& P,
                                         const C* __restrict__ stw, int tid0, int nthr, int nvalid = 0) {
  const int L = P.L;
  const int tid = (int)threadIdx.x - tid0;
  const bool mine = tid >= 0 && tid < nthr;
  for (int si = 0; si < P.nstages; ++si) {
    const int st = MODE == kInvDit ? P.nstages - 1 - si : si;
    const int Lb = P.blocklen[st];
    const unsigned mpl = P.magic_per_line[st], mM = P.magic_M[st];
    const C* tws = stw + P.stw_off[st];
    const bool prune = MODE == kFwdDif && si == 0 && nvalid > 0 && nvalid < L;
    if (mine) {
#define MM_STAGE(R)                                                                                    \
  case R:                                                                                              \
    if constexpr ((RSET & radix_bit(R)) != 0u) {                                                       \
      if (MODE == kInvDit) fft_stage<R, true, C>(buf, ldl, nlines, L, Lb, mpl, mM, tws, tid, nthr); \
      else if (MODE == kFwdDif && prune)                                                               \
        fft_stage<R, false, C, true>(buf, ldl, nlines, L, Lb, mpl, mM, tws, tid, nthr, nvalid);   \
      else if (MODE == kFwdDif)                                                                        \
        fft_stage<R, false, C>(buf, ldl, nlines, L, Lb, mpl, mM, tws, tid, nthr);                 \
      else fft_stage_dif_inv<R, C>(buf, ldl, nlines, L, Lb, mpl, mM, tws, tid, nthr);             \
    }                                                                                                  \
    break;
      switch (P.radix[st]) {
        MM_STAGE(2) MM_STAGE(3) MM_STAGE(4) MM_STAGE(5) MM_STAGE(6) MM_STAGE(8) MM_STAGE(9)
        MM_STAGE(10) MM_STAGE(12) MM_STAGE(15) MM_STAGE(16)
        default: break;
      }
#undef MM_STAGE
    }
    __syncthreads();
  }
}

// The quotient multiplier of the plan's per-stage divisors: n / d =
// __umulhi(n, fft_magic(d)) for n d < 2^32, 0 for d = 1 (no division); the
// same formula as the host planner's.
__host__ __device__ constexpr unsigned fft_magic(int d) {
  return d == 1 ? 0u : (unsigned)(0xFFFFFFFFull / (unsigned)d) + 1u;
}

// fft_smem for one plan known at compile time: three stages of radices R0, R1,
// R2 (first to last DIF stage, L = R0 R1 R2) on lines of stride LDL.  The
// same stage code with every length a constant, so the butterflies'
// shared-memory and twiddle offsets fold into the instructions (the results
// are those of fft_smem with the same plan, bit for bit).  The caller checks
// that P is this plan.  nvalid as for fft_smem (kFwdDif only).
template <int MODE, typename C, int R0, int R1, int R2, int LDL = R0 * R1 * R2>
__device__ __forceinline__ void fft_smem_fixed(C* buf, int nlines, const FftPlanDev& P,
                                               const C* __restrict__ stw, int tid0, int nthr, int nvalid = 0) {
  constexpr int L = R0 * R1 * R2;
  const int tid = (int)threadIdx.x - tid0;
  const bool mine = tid >= 0 && tid < nthr;
  // stage s: block length Lb, M = Lb / R butterfly stride, L / R butterflies
  // per line; the quotient multipliers are the planner's (fft_magic)
  constexpr int Lb0 = L, Lb1 = R1 * R2, Lb2 = R2;
  constexpr unsigned mpl0 = fft_magic(L / R0), mM0 = fft_magic(Lb0 / R0);
  constexpr unsigned mpl1 = fft_magic(L / R1), mM1 = fft_magic(Lb1 / R1);
  constexpr unsigned mpl2 = fft_magic(L / R2), mM2 = fft_magic(Lb2 / R2);
  const C* tw0 = stw + P.stw_off[0];
  const C* tw1 = stw + P.stw_off[1];
  const C* tw2 = stw + P.stw_off[2];
  if (MODE == kFwdDif) {
    if (mine) {
      if (nvalid > 0 && nvalid < L)
        fft_stage<R0, false, C, true>(buf, LDL, nlines, L, Lb0, mpl0, mM0, tw0, tid, nthr, nvalid);
      else
        fft_stage<R0, false, C>(buf, LDL, nlines, L, Lb0, mpl0, mM0, tw0, tid, nthr);
    }
    __syncthreads();
    if (mine) fft_stage<R1, false, C>(buf, LDL, nlines, L, Lb1, mpl1, mM1, tw1, tid, nthr);
    __syncthreads();
    if (mine) fft_stage<R2, false, C>(buf, LDL, nlines, L, Lb2, mpl2, mM2, tw2, tid, nthr);
    __syncthreads();
  } else if (MODE == kInvDit) {
    if (mine) fft_stage<R2, true, C>(buf, LDL, nlines, L, Lb2, mpl2, mM2, tw2, tid, nthr);
    __syncthreads();
    if (mine) fft_stage<R1, true, C>(buf, LDL, nlines, L, Lb1, mpl1, mM1, tw1, tid, nthr);
    __syncthreads();
    if (mine) fft_stage<R0, true, C>(buf, LDL, nlines, L, Lb0, mpl0, mM0, tw0, tid, nthr);
    __syncthreads();
  } else {
    if (mine) fft_stage_dif_inv<R0, C>(buf, LDL, nlines, L, Lb0, mpl0, mM0, tw0, tid, nthr);
    __syncthreads();
    if (mine) fft_stage_dif_inv<R1, C>(buf, LDL, nlines, L, Lb1, mpl1, mM1, tw1, tid, nthr);
    __syncthreads();
    if (mine) fft_stage_dif_inv<R2, C>(buf, LDL, nlines, L, Lb2, mpl2, mM2, tw2, tid, nthr);
    __syncthreads();
  }
}

// The plans with compile-time builds: 1 = 2160 = 16 9 15 and 3 = 540 = 4 9 15
// (the stick-slip grid's x and y), 2 = 1080 = 12 6 15 (the 512 x 512 films').
template <int ID> struct FixedPlan;
template <> struct FixedPlan<1> { static constexpr int R0 = 16, R1 = 9, R2 = 15, L = 2160; };
template <> struct FixedPlan<2> { static constexpr int R0 = 12, R1 = 6, R2 = 15, L = 1080; };
template <> struct FixedPlan<3> { static constexpr int R0 = 4, R1 = 9, R2 = 15, L = 540; };

// the id of P among the fixed plans, 0 if none
inline int fixed_plan_id(const FftPlanDev& P) {
  if (P.nstages != 3) return 0;
  const int r0 = P.radix[0], r1 = P.radix[1], r2 = P.radix[2];
  if (P.L == 2160 && r0 == 16 && r1 == 9 && r2 == 15) return 1;
  if (P.L == 1080 && r0 == 12 && r1 == 6 && r2 == 15) return 2;
  if (P.L == 540 && r0 == 4 && r1 == 9 && r2 == 15) return 3;
  return 0;
}

// fft_smem_fixed for fixed plan ID on lines of stride LDL
template <int MODE, int ID, int LDL, typename C>
__device__ __forceinline__ void fft_smem_plan(C* buf, int nlines, const FftPlanDev& P, const C* __restrict__ stw,
                                              int tid0, int nthr, int nvalid = 0) {
  typedef FixedPlan<ID> F;
  fft_smem_fixed<MODE, C, F::R0, F::R1, F::R2, LDL>(buf, nlines, P, stw, tid0, nthr, nvalid);
}

// Position of frequency k in the DIF output: sum_s M_s digit_s(k).
__device__ __forceinline__ int fft_pos(int k, const FftPlanDev& P) {
  int p = 0;
  for (int s = 0; s < P.nstages; ++s) {
    const int r = P.radix[s];
    const int q = (int)__umulhi((unsigned)k, P.magic_r[s]);
    p += (P.blocklen[s] / r) * (k - q * r);
    k = q;
  }
  return p;
}

// Frequency held at DIF position p (inverse of fft_pos).
__device__ __forceinline__ int fft_freq(int p, const FftPlanDev& P) {
  int k = 0, mult = 1;
  for (int s = 0; s < P.nstages; ++s) {
    const int M = P.blocklen[s] / P.radix[s];
    const int d = P.magic_M[s] ? (int)__umulhi((unsigned)p, P.magic_M[s]) : p;
    p -= d * M;
    k += mult * d;
    mult *= P.radix[s];
  }
  return k;
}

// Mirror (whole-sample symmetric) reflection of index j into [0, b).
__device__ __forceinline__ int mirror_index(int j, int b) {
  if (b <= 1) return 0;
  const int P = 2 * b - 2;
  j %= P;
  if (j < 0) j += P;
  return j < b ? j : P - j;
}

__device__ __forceinline__ int wrap_index(long long j, int Q) {
  long long m = j % Q;
  return (int)(m < 0 ? m + Q : m);
}

// j mod Q for -Q <= j < 2Q (box-local nodes never wrap more than once)
__device__ __forceinline__ int wrap_once(int j, int Q) { return j < 0 ? j + Q : (j >= Q ? j - Q : j); }

}  // namespace mm
