// Stray field from a caller-held coefficient box without any device allocation.
//
// Some callers cannot allocate device memory while they drive this library:
// an application whose device memory is entirely owned by its own pool
// allocator (a framework's caching allocator, a fixed-budget arena) and that
// forbids raw cudaMalloc, or a time-stepping loop in which the implicit device
// synchronisation of cudaMalloc / cudaFree would stall other streams.  For them
// mm_spline_field_noalloc runs the tricubic gather of the stray field and the
// force / energy reduction with its scratch (the per-tile partial sums,
// the displacement and an error flag) in the fixed array below, which every
// GPU that loads the library holds until the process exits.
//
// Set-up: the device address of the array is looked up with
// cudaGetSymbolAddress on the first call made on each device (with that
// device current) and cached; that first call should come before any stream
// capture.  Every call shares the one array per device: calls whose work
// overlaps on the GPU race on it, so serialise them (one stream, or events).
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "dfloat.cuh"
#include "mm.h"
#include "mm_internal.h"

namespace mm {

constexpr int kNoAllocMaxTiles = 65536;  // 32 x 8 target columns per tile -> 16.7M columns
constexpr int kNoAllocHeader = 32;       // [0] error flag, [1..3] displacement, [4..6] its cell,
                                         // [7..9] its fraction, rest spare
constexpr int kNoAllocMaxDevices = 64;

// 2 MiB: header + 4 doubles per gather tile
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocHeader + 4 * kNoAllocMaxTiles];

// Writes the displacement of the call into the scratch and clears the error flag.
__global__ void k_noalloc_begin(double p0, double p1, double p2) {
  if (threadIdx.x == 0) {
    reinterpret_cast<int*>(g_noalloc_scratch)[0] = 0;
    g_noalloc_scratch[1] = p0;
    g_noalloc_scratch[2] = p1;
    g_noalloc_scratch[3] = p2;
    int ucell[2][3];
    float ufrac[2][3];
    split_displacement(g_noalloc_scratch + 1, ucell, ufrac);
    for (int a = 0; a < 3; ++a) {
      reinterpret_cast<int*>(g_noalloc_scratch + 4)[a] = ucell[0][a];
      reinterpret_cast<float*>(g_noalloc_scratch + 7)[a] = ufrac[0][a];
    }
  }
}

// Fixed-order reduction of the tile partials into F[3], E (caller memory).
__global__ void __launch_bounds__(256) k_noalloc_reduce(int ntiles, double Fscale, double Escale,
                                                        double* FE_out) {
  __shared__ dfloat sh[8][4];
  // tile partials: [tile][4] double-float pairs
  const float2* part = reinterpret_cast<const float2*>(g_noalloc_scratch + kNoAllocHeader);
  dfloat v[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
    for (int c = 0; c < 4; ++c) {
      const float2 q = part[(size_t)t * 4 + c];
      v[c] = df_add(v[c], dfloat{q.x, q.y});
    }
  for (int c = 0; c < 4; ++c)
    for (int o = 16; o > 0; o >>= 1) v[c] = df_add(v[c], df_shfl_down(v[c], o));
  if ((threadIdx.x & 31) == 0)
    for (int c = 0; c < 4; ++c) sh[threadIdx.x >> 5][c] = v[c];
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[4];
    for (int c = 0; c < 4; ++c) {
      dfloat a = {0.f, 0.f};
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a = df_add(a, sh[w][c]);
      s[c] = df_to_double(a);
    }
    const int err = reinterpret_cast<const int*>(g_noalloc_scratch)[0];
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int c = 0; c < 3; ++c) FE_out[c] = err ? nan : Fscale * s[c];
    FE_out[3] = err ? nan : Escale * s[3];
  }
}

// Per-device address of the scratch array, looked up once with that device current.
static double* scratch_address(cudaError_t* err) {
  static std::mutex mu;
  static double* addr[kNoAllocMaxDevices] = {};
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return nullptr;
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    double* p = nullptr;
    *err = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (*err != cudaSuccess) return nullptr;
    addr[dev] = p;
  }
  return addr[dev];
}

}  // namespace mm

using namespace mm;

extern "C" mm_status mm_spline_field_noalloc(const float* coef_dev, const int coef_dims[3],
                                             const long long coef_lo[3], const double pos0_nodes[3],
                                             const float* m_dev, int nx, int ny, int nz, double dx,
                                             double dy, double dz, double Ms, float* H_dev,
                                             double* FE_dev, void* stream) {
  if (!coef_dev || !coef_dims || !coef_lo || !pos0_nodes || !m_dev || !FE_dev) return MM_EINVAL;
  if (nx < 1 || ny < 1 || nz < 1 || nz > kMaxNz || !(dx > 0) || !(dy > 0) || !(dz > 0) || !(Ms > 0))
    return MM_EINVAL;
  // positions beyond 2^30 nodes would overflow the int lattice indices of the gather
  for (int a = 0; a < 3; ++a)
    if (coef_dims[a] < 4 || !isfinite(pos0_nodes[a]) || fabs(pos0_nodes[a]) >= 1073741824.0 ||
        coef_lo[a] <= -(1ll << 40) || coef_lo[a] >= (1ll << 40))
      return MM_EINVAL;
  // tile count in 64 bits: a huge nx * ny must not wrap below the limit
  const long long ntiles_ll = ((long long)nx + 31) / 32 * (((long long)ny + 7) / 8) *
                              (((long long)nz + kMaxNz - 1) / kMaxNz);
  if (ntiles_ll > kNoAllocMaxTiles) return MM_ETOOBIG;
  const int ntiles = gather_tiles(nx, ny, nz);
  // support of every target centre must lie inside the coefficient box
  const int n[3] = {nx, ny, nz};
  GatherJob J{};
  for (int a = 0; a < 3; ++a) {
    const double fl = floor(pos0_nodes[a]);
    const long long first = (long long)fl - 1 - coef_lo[a];  // coefficient index of the first tap
    if (first < 0 || first + n[a] + 3 > coef_dims[a]) return MM_ERANGE;
    J.U0[a] = (int)fl;
    J.guard[a] = (int)first;
  }
  cudaError_t e;
  double* scratch = scratch_address(&e);
  if (!scratch) return MM_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  k_noalloc_begin<<<1, 32, 0, st>>>(pos0_nodes[0], pos0_nodes[1], pos0_nodes[2]);
  if ((e = cudaGetLastError()) != cudaSuccess) return MM_ECUDA;
  J.C = coef_dev;
  J.rx = coef_dims[0]; J.ry = coef_dims[1]; J.rz = coef_dims[2];
  J.nx = nx; J.ny = ny; J.nz = nz;
  J.ucell = reinterpret_cast<const int*>(scratch + 4);
  J.ufrac = reinterpret_cast<const float*>(scratch + 7);
  J.inv_d[0] = (float)(1.0 / dx);
  J.inv_d[1] = (float)(1.0 / dy);
  J.inv_d[2] = (float)(1.0 / dz);
  J.m = m_dev;
  J.H = H_dev;
  J.partial = reinterpret_cast<float2*>(scratch + kNoAllocHeader);
  J.err = reinterpret_cast<int*>(scratch);
  Launch<GatherJob> L{};
  L.njobs = 1;
  L.tile_start[0] = 0;
  L.tile_start[1] = ntiles;
  L.job[0] = J;
  // tile partials only; k_noalloc_reduce below sums them
  if (launch_gather(L, nz, st) != cudaSuccess) return MM_ECUDA;
  const double mu0 = 4e-7 * 3.14159265358979323846;
  const double V = dx * dy * dz;
  k_noalloc_reduce<<<1, 256, 0, st>>>(ntiles, -mu0 * V * Ms, mu0 * V * Ms, FE_dev);
  if (cudaGetLastError() != cudaSuccess) return MM_ECUDA;
  return MM_OK;
}
