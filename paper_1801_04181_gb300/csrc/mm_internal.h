// Internal types shared by the CUDA translation units of libmm.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mm {

constexpr int kMaxStages = 16;
constexpr int kMaxJobs = 4;        // jobs per launch (two magnets / two directions)
constexpr int kFirHalf = 14;       // B-spline prefilter FIR half-width, |z1|^15 ~ 2.6e-9
constexpr int kMaxNz = 4;          // thin-film path: z handled by direct plane mixing
constexpr int kMaxOut = kMaxNz + 5; // coefficient planes: nz + 3 + 2 guard
constexpr int kRowsPerCta = 8;     // real rows per CTA in the x passes (4 complex lines)

// FFT radix sets: one bit per radix the shared-memory FFT implements
__host__ __device__ constexpr unsigned radix_bit(int R) {
  return R == 2 ? 1u : R == 3 ? 2u : R == 4 ? 4u : R == 5 ? 8u : R == 6 ? 16u : R == 8 ? 32u
       : R == 9 ? 64u : R == 10 ? 128u : R == 12 ? 256u : R == 15 ? 512u : R == 16 ? 1024u : 0u;
}
constexpr unsigned kAllRadices = 2047u;
// the set the FFT pass kernels are also built for: {4, 9, 15, 16} (every length
// 4^a 9^b 15^c 16^d, among them 540 = 4 9 15 and 2160 = 16 9 15)
constexpr unsigned kRadixSetA = 4u | 64u | 512u | 1024u;

struct FftPlanDev {
  int L;
  int nstages;
  int radix[kMaxStages];
  int blocklen[kMaxStages];
  // n / d = __umulhi(n, magic) for the two per-stage divisors (L / r and
  // Lb / r); exact while n * d < 2^32, which holds for every launch here
  unsigned magic_per_line[kMaxStages];
  unsigned magic_M[kMaxStages];
  unsigned magic_r[kMaxStages];
  // stage twiddle table s starts at entry stw_off[s] of FftTables::tw_f / tw_d:
  // W_Lb^{n1 k} at (k - 1) M + n1, M = blocklen / radix, k = 1 .. radix - 1
  int stw_off[kMaxStages];
};

// Length-L transform resources resident on the device.
struct FftTables {
  FftPlanDev plan;
  const float2* tw_f;     // stage twiddle tables, W_Lb^{n1 k} (see FftPlanDev)
  const double2* tw_d;
  const int* pos;         // frequency k -> position in DIF output
  const int* freq;        // position -> frequency
};

// ---------------------------------------------------------------- x forward
struct XFwdJob {
  const float* m;         // [3][nz][ny][nx]
  float2* out;            // [3 nz][kxh][ny]
  int nx, ny, nz;
  int kxh;
  FftTables fx;
  // reduced precision: the rows (plane, kx) written split into BF16 hi | lo
  // blocks for the forward y DFT (ceil(ny / 16) K chunks) instead of `out`
  uint16_t* pk;
};

// ---------------------------------------------------------------- y pass
struct YJob {
  const float2* in;       // [3 nz][kxh][ny]
  int nz, ny, kxh;
  FftTables fy;
  int kyq;                // Qy/2 + 1 stored ky values of the kernel spectra
  // self-demag output
  int do_H;
  const float* Nq;        // [6][nz][kxh][kyq]  (xx yy zz xy xz yz; dz >= 0)
  float2* outH;           // [3 nz][kxh][ny]
  // potential / coefficient output
  int do_C;
  int n_out;
  const float* Tq;        // [n_out][nz][3][kxh][kyq]
  float2* outC;           // [n_out][kxh][r]
  int box_lo, box_len, start, r, fir;
  int periodic;           // the y box is the whole period: the prefilter wraps
};

// ---------------------------------------------------------------- x inverse
struct XInvJob {
  const float2* in;       // [planes][kxh][rows_per_plane]
  float* out;             // [planes][rows_per_plane][out_len]
  int planes, rows_per_plane, kxh;
  FftTables fx;
  // output window along x: circular index (box_lo + j) mod Q for box-local j
  int box_lo, box_len, start, out_len, fir;
  int periodic;           // the x box is the whole period: the prefilter wraps
};

// ---------------------------------------------------------------- 3D sources (nz > kMaxNz)
// y FFT of X1 columns; out[kx][pos][plane], positions in the plan's DIF order
struct YFwdJob {
  const float2* in;       // [planes][kxh][ny]
  float2* out;            // natural = 0: [kxh][Qy][planes], DIF positions
                          // natural = 1: [planes][kxh][Qy], frequencies in natural order
  int planes, ny, kxh;
  int group;              // planes per CTA
  int natural;
  FftTables fy;
};

// z FFT, spectral products, inverse z FFT and z prefilter for a tile of y positions
struct ZJob {
  const float2* in;       // [kxh][Qy][3 nz]
  int nz, kxh;
  FftTables fy, fz;       // fy: frequency of a y position; fz: the z transforms
  int kyq, kzq;           // stored ky <= Qy/2, kz <= Qz/2
  const float* N3;        // [6][kxh][kyq][kzq], -Ms N / (Qx Qy Qz)
  const float* S3;        // [3][kxh][kyq][kzq], imaginary parts of Ms S / (Qx Qy Qz)
  int do_H, do_C;
  float2* outH;           // [3 nz][kxh][Qy]
  float2* outC;           // [r][kxh][Qy]
  int box_lo, box_len, start, r, fir;  // z box of the coefficient planes
  int ztile;              // y positions per CTA
};

// inverse y FFT (DIF-order positions in, natural out) and the y outputs
struct YInvJob {
  const float2* in;       // [planes][kxh][Qy], DIF positions (natural = 0) or frequencies (1)
  int natural;
  int planes, kxh;
  int group;
  FftTables fy;
  int is_C;               // 0: demag rows y < ny -> outH; 1: coefficient rows -> outC
  int ny;
  float2* outH;           // [planes][kxh][ny]
  float2* outC;           // [planes][kxh][r]
  int box_lo, box_len, start, r, fir;  // y box
  int periodic;           // the y box is the whole period: the prefilter wraps
};

// direct z sum for moderately thick sources (nz <= kMaxNzDirect): thin-film
// style plane mixing between the y-forward and y-inverse passes, ky natural
struct ZMixJob {
  const float2* in;       // [3 nz][kxh][Qy]
  int nz, kxh, Qy, kyq;
  const float* Nq;        // [6][nz][kxh][kyq]
  const float* Tq;        // [n_out][nz][3][kxh][kyq]
  int nH, n_out;          // output planes: 3 nz demag (if nH), then n_out coefficient planes
  float2* outH;           // [3 nz][kxh][Qy]
  float2* outC;           // [n_out][kxh][Qy]
  // 0: potential planes (Tq of S); > 0: the componentwise field variant, whose
  // n_out = 3 field_nbox planes are H_a of box plane o at a field_nbox + o,
  // with Tq the W-folded rows of -N (build_TN_spectra)
  int field_nbox;
  // reduced precision: outputs written split into BF16 hi | lo blocks for the
  // inverse DFT (rows (plane, kx), ceil(Qy / 16) K chunks) instead of outH / outC
  uint16_t* pkH;
  uint16_t* pkC;
};
constexpr int kMaxNzDirect = 8;

// ---------------------------------------------------------------- reduced-precision y stage
// y transforms as DFT-matrix products on the tensor cores (csrc/ydft.cu):
// D[row][0:Nc] = sum_k A[row][k] F(k, .), complex rows of one (plane, kx)
// line each; F in real form, split into BF16 hi + lo parts and packed in the
// tensor core's no-swizzle K-major layout, [ntiles][kchunks][ntile x 64].
enum DftKind { kDftForward = 0, kDftInverse = 1, kDftInversePrefilter = 2 };
constexpr int kDftPrefTaps = 24;  // prefilter taps each side: |z1|^24 ~ 2e-14
struct DftSpec {                  // what a packed matrix holds (compared bytewise)
  int kind;
  int Q;                          // y grid length
  int Nc, Kc;                     // complex outputs / inputs per row
  int box_lo, box_len, start;     // kDftInversePrefilter: the y box and the first row
  int periodic, fir;              // wrapped box; prefilter on (else plain node values)
};
struct DftShape {
  int ntile = 0;                  // real output columns per CTA (a multiple of 16, <= 160)
  int ntiles = 0;
  int kchunks = 0;                // K chunks of 64 real values
};
struct DftJob {
  const float2* A;                // [rows][lda], the first Kc of a row used
  int lda, rows, Kc;
  uint16_t* Apk;                  // A split into BF16 hi | lo, packed per (128-row tile, K chunk),
                                  // written by the pass that produces A (store_split)
  const uint16_t* Bhi;
  const uint16_t* Blo;
  int ntile, ntiles, kchunks, Nc;
  float2* D;                      // [rows][ldd], the first Nc written
  int ldd;
  int* err;                       // bit 2 set when a wait on the tensor core ran out
};

// ---------------------------------------------------------------- adjoint (energy gradients)
// transposed gradient evaluation: coefficient-region node n collects
// escale * m_t,a(i) / d_a * (derivative weights of axis a) from the targets i
// whose 64 taps cover it; written into the box at offset `start`
struct AdjScatterJob {
  const float* m;         // target unit magnetisation [3][N]
  int nx, ny, nz;         // target grid
  const double* u;        // slider displacement, lattice cells (device)
  double sigma;
  int U0[3], guard[3];
  float inv_d[3];
  float escale;           // mu0 V Ms_t
  float* box;             // [bz][by][bx]
  int bdim[3];            // box extents
  int start[3];           // coefficient region inside the box
  int r[3];               // coefficient region extents
  int* err;
};

// transposed potential sum in the spectral domain (direct z): for source
// plane (c, jz), sum over box planes zb of conj(S_c(zb - jz)) phibar(zb)
struct ZAdjJob {
  const float2* in;       // [bz][kxh][Qy], ky natural
  int bz, nz, kxh, Qy, kyq;
  const float* Sq;        // [bz + nz - 1][3][kxh][kyq]: quarter spectra per z offset, scaled
  float2* out;            // [3 nz][kxh][Qy]
};

// ---------------------------------------------------------------- gather
struct GatherJob {
  const float* C;         // coefficients [rz][ry][rx]
  int rx, ry, rz;
  int nx, ny, nz;         // target grid
  const int* ucell;       // floor(sigma u) per axis (device), u the slider displacement in lattice cells
  const float* ufrac;     // sigma u - floor(sigma u) per axis (device)
  int U0[3];              // floor(sigma u) when the box was planned
  int guard[3];           // extra coefficient nodes kept on each side
  float inv_d[3];         // 1 / cell size (1/m)
  const float* m;         // target unit magnetisation [3][N]
  float* H;               // stray field out [3][N] (A/m), may be null
  float2* partial;        // [tiles][4] double-float (hi, lo): sum m.Hess (3), sum m.grad
  int* err;               // set to 1 when the displacement leaves the box
  // periodic x (a = 0), y (a = 1): the coefficients span the period wrapP[a]
  // from source node 0, and the first tap of target cell i is node
  // tap0[a] + floor(sigma u_a) + i (mod the period); 0 = open axis
  int wrapP[2], tap0[2];
};

// ---------------------------------------------------------------- LLG / RK
struct StageJob {
  const float* ys;        // stage input m [3][N]
  const float* y;         // accepted state [3][N]
  float* ys_next;         // next stage input
  float* k[7];            // stage derivatives
  const float* Hself;
  const float* Hstray;
  const float* Heddy;     // eddy field of a conducting magnet (A/m), null if none
  float* Heff;            // optional effective field out
  int nx, ny, nz;
  float ex[3];            // 2 A / (mu0 Ms d_a^2)
  float an;               // 2 Ku / (mu0 Ms)
  float ku[3];            // unit easy axis
  float hext[3];
  float pref;             // -gamma0 / (1 + alpha^2)
  float alpha;
  int stage;              // 1..7
  int mode;               // 0 RK stage, 1 right-hand side only
  float comb[7];          // dt a_{stage+1, j}
  float ecoef[7];         // dt (b5_j - b4_j)
  float* err_partial;     // per-CTA max |error| (stage 7)
  int wrap[2];            // exchange neighbours wrap around x (0), y (1): periodic boundaries
};

struct CombineJob {
  const float* y;
  float* out;
  const float* k[7];
  float comb[7];
  int nk;
  size_t n;               // cells
};

struct MechState {
  double x, v, t;         // accepted slider position (m), velocity, time
  double xs, vs, ts;      // current stage values
  double kx[7], kv[7];
  double u[3];            // displacement (lattice cells) seen by the gathers
  double F_slider[3], E_slider, F_base[3], E_base;
  double err;
  // u split for the gathers, row 0 for sigma = +1 (target is the slider) and
  // row 1 for sigma = -1: floor(sigma u) and sigma u - floor(sigma u)
  int ucell[2][3];
  float ufrac[2][3];
};

// The integer and fractional lattice offsets of both directions (FP64 floor,
// the fraction exact in FP64 and then rounded to float), on the host or in the
// one thread that writes u.
__host__ __device__ inline void split_displacement(const double* u, int (*ucell)[3], float (*ufrac)[3]) {
  for (int r = 0; r < 2; ++r)
    for (int a = 0; a < 3; ++a) {
      const double su = r == 0 ? u[a] : -u[a];
      const double fl = floor(su);
      ucell[r][a] = (int)fl;
      ufrac[r][a] = (float)(su - fl);
    }
}

struct MechParams {
  MechState* state;
  const float2* partial[2];   // gather tile partials [nparts][4] (hi, lo): [0] base -> slider, [1] slider -> base
  int nparts[2];
  double Fscale[2], Escale[2];
  const float* err_partial[2];
  int nerr[2];
  int mode;               // 0 RK stage, 1 forces only, 2 stage-2 input from k1, 3 accept,
                          // 4 restart, 5 error norm of the attempt
  int stage;
  double dt;
  double a[7];            // a_{stage+1, j}
  double c_next;
  int move;               // slider equation of motion active
  double mass, inv_mass, k_spring, v_drive, x0_spring, gamma_v;
  double e[3], inv_d[3], u_base[3];
};

template <typename J> struct Launch {
  int njobs;
  int tile_start[kMaxJobs + 1];
  J job[kMaxJobs];
};

__device__ __forceinline__ int find_job(const int* tile_start, int njobs, int tile) {
  int j = 0;
  while (j + 1 < njobs && tile >= tile_start[j + 1]) ++j;
  return j;
}

}  // namespace mm

// ---------------------------------------------------------------- host entry points
namespace mm {

struct KernelPlan {
  int Qx, Qy;             // circular grid
  int Wx, Wy;             // kernel window |d| <= W (cells)
  int nz;                 // source layers
  int px = 0, py = 0;     // periodic axis: Q is the period, every offset counts, images summed
  int R = 0;              // periodic images on each side
};

struct KernelPlan3 {
  int Qx, Qy, Qz;
  int Wx, Wy, Wz;
};

cudaError_t init_fft_constants_passes();
cudaError_t init_fft_constants_kgen();
cudaError_t init_fft_constants_3d();
size_t ypass_table_bytes(int r);
cudaError_t launch_xfwd(const Launch<XFwdJob>& L, int Qmax, cudaStream_t st);
cudaError_t launch_ypass(const Launch<YJob>& L, size_t smem, cudaStream_t st);
cudaError_t launch_xinv(const Launch<XInvJob>& L, int Qmax, cudaStream_t st);
cudaError_t launch_yfwd3(const Launch<YFwdJob>& L, cudaStream_t st);
cudaError_t launch_zpass3(const Launch<ZJob>& L, cudaStream_t st);
cudaError_t launch_yinv3(const Launch<YInvJob>& L, cudaStream_t st);
cudaError_t launch_zmix3(const Launch<ZMixJob>& L, cudaStream_t st);
DftShape dft_shape(int Nc, int Kc);
size_t dft_matrix_elems(const DftShape& s);
int dft_tiles(int rows, const DftShape& s);
size_t dft_a_bytes(int rows, const DftShape& s);  // a packed split operand
cudaError_t launch_dft_pack(const DftSpec& P, const DftShape& s, uint16_t* hi, uint16_t* lo, cudaStream_t st);
cudaError_t launch_ydft(const Launch<DftJob>& L, cudaStream_t st);
cudaError_t launch_adj_scatter(const AdjScatterJob& J, cudaStream_t st);
cudaError_t launch_pref_T(float* box, const int bdim[3], cudaStream_t st);
cudaError_t launch_place(const float* box, const int bdim[3], const int box_lo[3], float* grid, int Qx, int Qy,
                         cudaStream_t st);
cudaError_t launch_zadj(const ZAdjJob& J, cudaStream_t st);
cudaError_t launch_scale(const float* in, float* out, size_t n, float s, cudaStream_t st);

// power bookkeeping (power.cu): *out = sum_i |m_i x H_i|^2 over N cells;
// partial holds power_blocks(N) doubles
int power_blocks(size_t N);
cudaError_t launch_mxh2(const float* m, const float* H, size_t N, double* partial, double* out, cudaStream_t st);
// four-point difference gradient of the interpolant (variants.cu): V holds
// (nx + 4)(ny + 4)(nz + 4) floats, H 3 nx ny nz; needs margin >= 2
// eddy currents (eddy.cu)
cudaError_t launch_cross_input(const float* V, size_t N, int comp, float* out, cudaStream_t st);
cudaError_t launch_scale_into(const float* in, size_t N, float s, float* out, cudaStream_t st);
cudaError_t launch_accumulate(const float* in, size_t N, float* out, cudaStream_t st);  // out += in
int eddy_blocks(size_t N);
cudaError_t launch_eddy_source(const float* E, int nx, int ny, int nz, const double d[3], double* b, double* part,
                               double* bmean, cudaStream_t st);
cudaError_t launch_sor_sweeps(double* phi, const double* b, const double* bmean, int nx, int ny, int nz,
                              const double d[3], double omega, int sweeps, cudaStream_t st);
cudaError_t launch_sor_residual(const double* phi, const double* b, const double* bmean, int nx, int ny, int nz,
                                const double d[3], double* part, double* stats, cudaStream_t st);
cudaError_t launch_eddy_current(const double* phi, const double* stats, const float* E, int nx, int ny, int nz,
                                const double d[3], double sigma, float* J, cudaStream_t st);
cudaError_t launch_flux_rate(const float* Hself, const float* Hstray, const float* y, size_t N, const double hext[3],
                             double Ms, double dt, int have_prev, float* Bprev, float* Bdot, cudaStream_t st);

// componentwise field variant (variants.cu): H_a at every target centre from
// the coefficients C [3][bdim z][bdim y][bdim x] of the three components on
// the full box (taps of centre i start at node i + margin)
cudaError_t launch_field_values(const float* C, const int bdim[3], const int nt[3], int margin,
                                const double frac[3], float* H, cudaStream_t st);
cudaError_t launch_fd4_field(const float* C, const int bdim[3], const int nt[3], int margin, const double frac[3],
                             const double cell[3], float* V, float* H, cudaStream_t st);

// div / curl means (power.cu): out[0] = sum |div H|, out[1] = sum ||curl H|| over
// divcurl_cells interior cells; partial holds 2 divcurl_blocks doubles
size_t divcurl_cells(int nx, int ny, int nz);
int divcurl_blocks(int nx, int ny, int nz);
cudaError_t launch_divcurl(const float* H, int nx, int ny, int nz, double dx, double dy, double dz,
                           double* partial, double* out, cudaStream_t st);
int zmix_tiles(int kyq, int planes);
int zpass_tile(int Qz);                 // y positions per z-pass CTA for a z grid
int zpass_tiles(int Qy, int ztile);
int gather_tiles(int nx, int ny, int nz);  // 32 x 8 columns x up to kMaxNz layers
size_t gather_smem(int nz);
cudaError_t launch_gather(const Launch<GatherJob>& L, int nz_max, cudaStream_t st);
cudaError_t launch_stage(const Launch<StageJob>& L, const MechParams& Perr, int* ticket, cudaStream_t st);
cudaError_t launch_combine(const Launch<CombineJob>& L, cudaStream_t st);
cudaError_t launch_normalise(const Launch<CombineJob>& L, cudaStream_t st);
cudaError_t launch_mech(const MechParams& P, cudaStream_t st);
cudaError_t eval_points_fp64(int kind, int n, const double* off_dev, double a, double b, double c,
                             double* out_dev, cudaStream_t st);
cudaError_t build_N_spectra(const KernelPlan& K, const FftTables& fx, const FftTables& fy, double a,
                            double b, double c, double scale, float* Nq, double2* work, double* qbuf,
                            cudaStream_t st);
// 3D spectra of S (kind 0, 3 comps) or N (kind 1, 6 comps): out [comp][kxh][kyq][kzq].
// Scratch: work 2 * ncomp * Qx * Qy double2, q2 ncomp * Qz * kxh * kyq double,
// qtmp ncomp * kxh * kyq double, zl kxh * kyq * Qz double2.
cudaError_t build_spectra_3d(int kind, const KernelPlan3& K, const FftTables& fx, const FftTables& fy,
                             const FftTables& fz, double a, double b, double c, double scale, float* out,
                             double2* work, double* q2, double* qtmp, double2* zl, cudaStream_t st);
// FP32 quarter spectra of S, one plane of 3 components per z offset dz_lo + p,
// p < nplanes: Sq [p][3][kxh][kyq], scaled.  work as for build_N_spectra,
// qtmp 3 kxh kyq doubles.
// Componentwise field variant: TN [3][n_out][nz][3][kxh][kyq], the rows of N
// folded with the z mixing matrix W, scaled.  Nq6 scratch (bz + nz - 1) 6 kxh kyq
// doubles, work as for build_N_spectra.
cudaError_t build_TN_spectra(const KernelPlan& K, const FftTables& fx, const FftTables& fy, double a,
                             double b, double c, double scale, int box_lo_z, int bz, int n_out,
                             const double* W_dev, float* TN, double2* work, double* Nq6, cudaStream_t st);
cudaError_t build_S_planes(const KernelPlan& K, const FftTables& fx, const FftTables& fy, double a, double b,
                           double c, double scale, int dz_lo, int nplanes, float* Sq, double2* work,
                           double* qtmp, cudaStream_t st);
cudaError_t build_T_spectra(const KernelPlan& K, const FftTables& fx, const FftTables& fy, double a,
                            double b, double c, double scale, int box_lo_z, int bz, int n_out,
                            const double* W_dev, float* Tq, double2* work, double* Sq,
                            cudaStream_t st);

}  // namespace mm
