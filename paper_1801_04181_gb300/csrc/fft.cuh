// Shared-memory mixed-radix FFT core (radix 2, 3, 4, 5, 8), in place.
//
// Forward transforms run decimation-in-frequency stages: natural-order input,
// output left in the mixed-radix digit-reversed order of the plan (frequency k
// sits at position pos[k]).  Inverse transforms run the exact stage inverses
// in reverse order: digit-reversed input, natural-order output, unnormalised
// (sum_k X[k] e^{+2 pi i n k / L}).  A forward + pointwise + inverse sequence
// therefore never needs a reordering pass.
//
// One stage of block length Lb = r * M maps, for every n1 < M,
//   x[n1 + M n2] -> y[k2] = W_Lb^{n1 k2} sum_n2 x[n1 + M n2] W_r^{n2 k2}
// stored back at n1 + M k2; twiddles come from a per-length table
// W_L[t] = exp(-2 pi i t / L) (index n1 k2 L / Lb < L).
#pragma once
#include <cuda_runtime.h>

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

// Small DFTs y[k] = sum_n x[n] exp(s 2 pi i n k / r), s = -1 forward, +1 inverse.
template <typename C> __device__ __forceinline__ void dft2(C* x) {
  C a = x[0], b = x[1];
  x[0] = cadd(a, b); x[1] = csub(a, b);
}
template <typename C> __device__ __forceinline__ void dft3(C* x, int s) {
  typedef typename cplx_traits<C>::real R;
  const R h = (R)0.86602540378443864676;  // sqrt(3)/2
  C t = cadd(x[1], x[2]);
  C m = csub(x[0], cscale(t, (R)0.5));
  C d = cscale(csub(x[1], x[2]), h);
  C id = cmul_is(d, s);
  x[0] = cadd(x[0], t);
  x[1] = cadd(m, id);
  x[2] = csub(m, id);
}
template <typename C> __device__ __forceinline__ void dft4(C* x, int s) {
  C a = cadd(x[0], x[2]), b = csub(x[0], x[2]);
  C c = cadd(x[1], x[3]), d = cmul_is(csub(x[1], x[3]), s);
  x[0] = cadd(a, c); x[2] = csub(a, c);
  x[1] = cadd(b, d); x[3] = csub(b, d);
}
template <typename C> __device__ __forceinline__ void dft5(C* x, int s) {
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
template <typename C> __device__ __forceinline__ void dft8(C* x, int s) {
  typedef typename cplx_traits<C>::real R;
  const R q = (R)0.70710678118654752440;  // 1/sqrt(2)
  C e[4] = {x[0], x[2], x[4], x[6]};
  C o[4] = {x[1], x[3], x[5], x[7]};
  dft4(e, s);
  dft4(o, s);
  // W8^k = exp(s 2 pi i k / 8)
  C w1o = cscale(cadd(o[1], cmul_is(o[1], s)), q);          // (1 + i s)/sqrt2
  C w2o = cmul_is(o[2], s);                                  // i s
  C w3o = cscale(csub(cmul_is(o[3], s), o[3]), q);          // (-1 + i s)/sqrt2
  x[0] = cadd(e[0], o[0]); x[4] = csub(e[0], o[0]);
  x[1] = cadd(e[1], w1o); x[5] = csub(e[1], w1o);
  x[2] = cadd(e[2], w2o); x[6] = csub(e[2], w2o);
  x[3] = cadd(e[3], w3o); x[7] = csub(e[3], w3o);
}

template <typename C> __device__ __forceinline__ void dft_small(C* x, int r, int s) {
  switch (r) {
    case 2: dft2(x); break;
    case 3: dft3(x, s); break;
    case 4: dft4(x, s); break;
    case 5: dft5(x, s); break;
    case 8: dft8(x, s); break;
    default: break;
  }
}

// Runs all stages of one transform on `nlines` lines of buf (line stride ldl),
// using the threads [tid0, tid0 + nthr) of the block.  The caller syncs before.
template <typename C>
__device__ void fft_smem(C* buf, int ldl, int nlines, const FftPlanDev& P, const C* __restrict__ tw,
                         bool inverse, int tid0, int nthr) {
  const int L = P.L;
  const int tid = (int)threadIdx.x - tid0;
  for (int si = 0; si < P.nstages; ++si) {
    const int st = inverse ? P.nstages - 1 - si : si;
    const int r = P.radix[st];
    const int Lb = P.blocklen[st];
    const int M = Lb / r;
    const int tstride = L / Lb;
    const int per_line = L / r;
    const int nb = nlines * per_line;
    if (tid >= 0 && tid < nthr) {
      for (int b = tid; b < nb; b += nthr) {
        const int line = b / per_line;
        const int rem = b - line * per_line;
        const int blk = rem / M;
        const int n1 = rem - blk * M;
        C* base = buf + (size_t)line * ldl + blk * Lb + n1;
        C v[8];
        if (!inverse) {
#pragma unroll
          for (int k = 0; k < 8; ++k) if (k < r) v[k] = base[k * M];
          dft_small(v, r, -1);
#pragma unroll
          for (int k = 1; k < 8; ++k)
            if (k < r) v[k] = cmul(v[k], tw[n1 * k * tstride]);
#pragma unroll
          for (int k = 0; k < 8; ++k) if (k < r) base[k * M] = v[k];
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) if (k < r) v[k] = base[k * M];
#pragma unroll
          for (int k = 1; k < 8; ++k)
            if (k < r) v[k] = cmulconj(v[k], tw[n1 * k * tstride]);
          dft_small(v, r, +1);
#pragma unroll
          for (int k = 0; k < 8; ++k) if (k < r) base[k * M] = v[k];
        }
      }
    }
    __syncthreads();
  }
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

}  // namespace mm
