// C ABI of libmm: planning, buffers and launch sequences (include/mm.h).
//
// Per source magnet s and target t = 1 - s (Sec. II.A: each magnet's stray
// field is interpolated inside the other):
//   box    per axis [floor(p_min) - 1 - margin, floor(p_max) + 2 + margin] in
//          source lattice nodes, p = offset_t - offset_s + i + sigma u
//          (Sec. III.A: potential extends `margin` cells past the support);
//   FFT    one Qx x Qy circular grid serves the magnet's own demag field and its
//          potential on the box: the kernels are laid on the window |d| <= W,
//          W covering every source-to-box offset, and Q >= 2W + 2 keeps the
//          circular sum equal to the linear one (no aliasing) and the kernels
//          exactly even / odd on the grid;
//   output coefficient nodes [margin - guard, margin + n_t + 3 + guard) per axis,
//          the spline support of all targets plus `guard` nodes on an axis of
//          motion so a step may cross a cell boundary without re-planning.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "mm.h"
#include "mm_internal.h"

using namespace mm;

namespace {

constexpr double kMu0 = 4e-7 * 3.14159265358979323846;
constexpr double kGammaLL = 1.7595e11;  // rad / (s T)
constexpr int kWindowSlack = 8;         // cells of displacement before the FFT grid is re-planned
constexpr int kTimingClasses = 10;
constexpr int kAttemptLog = 4096;  // step attempts the context remembers

// Dormand-Prince 5(4)
const double DP_C[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
const double DP_A[7][7] = {
    {0, 0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0}};
const double DP_B5[7] = {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0};
const double DP_B4[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200,
                         187.0 / 2100, 1.0 / 40};

struct FftRes {
  FftTables t{};
  float2* tw_f = nullptr;
  double2* tw_d = nullptr;
  int* pos = nullptr;
  int* freq = nullptr;
};

// a packed y-DFT matrix of the reduced-precision form and what it was built for
struct DftMat {
  uint16_t* hi = nullptr;
  uint16_t* lo = nullptr;
  size_t hi_bytes = 0, lo_bytes = 0;
  bool valid = false;
  DftSpec spec{};
  DftShape shape{};
};

struct Dir {
  bool valid = false;
  bool full_box = false;   // potential query: whole box, optional prefilter
  int prefilter = 1;
  int U0[3] = {0, 0, 0};
  int box_lo[3] = {0, 0, 0}, box_len[3] = {0, 0, 0};
  int start[3] = {0, 0, 0}, r[3] = {0, 0, 0}, guard[3] = {0, 0, 0};
  int Tq_box_lo_z = 0, Tq_bz = 0, Tq_start_z = 0, Tq_nout = 0, Tq_prefilter = -1, Tq_Q[2] = {0, 0};
  int Tq_kind = 0;             // 0: S (potential); 1: rows of -N (componentwise field variant)
  float* Tq = nullptr;
  float2* YC = nullptr;
  float* C = nullptr;
  float2* partial = nullptr;   // gather tile partials [ntiles][4], double-float
  int ntiles = 0;
  float2* Z3C = nullptr;       // thick sources: z-pass coefficient planes [r_z][kxh][Qy]
  size_t Tq_bytes = 0, YC_bytes = 0, C_bytes = 0, partial_bytes = 0, Z3C_bytes = 0;
  DftMat yiC;                  // reduced precision: inverse y DFT with the y prefilter
  uint16_t* pkC = nullptr;     // reduced precision: z-mixed coefficient planes, split and packed
  size_t pkC_bytes = 0;
  long long pkC_key = -1;
};

struct Magnet {
  bool grid = false, mat = false, mset = false;
  int nx = 0, ny = 0, nz = 0;
  long long off[3] = {0, 0, 0};
  double d[3] = {0, 0, 0};
  double Ms = 0, Aex = 0, Ku = 0, ku[3] = {0, 0, 1}, alpha = 0;
  size_t N = 0;
  float* m = nullptr;
  float* ys[2] = {nullptr, nullptr};
  float* k[7] = {};
  float* Hself = nullptr;
  float* Hstray = nullptr;
  float* scratch3 = nullptr;  // 3N scratch for rhs-only evaluations
  // power bookkeeping (allocated on first use): H_eff, block sums, the sum
  float* pow_H = nullptr;
  size_t pow_H_bytes = 0;
  double* pow_part = nullptr;
  size_t pow_part_bytes = 0;
  float* err_partial = nullptr;
  int nerr = 0;
  // as a source
  int Qx = 0, Qy = 0, Wx = 0, Wy = 0, kxh = 0, kyq = 0;
  double Nq_Ms = 0;
  float2* X1 = nullptr;
  float2* YH = nullptr;
  float* Nq = nullptr;
  // thick sources (y-forward, z and y-inverse passes): z by a direct sum over
  // planes (zfft false, nz <= kMaxNzDirect; spectra Nq and Tq as for thin
  // films) or by FFT (grid depth, spectra N3 / S3)
  bool thick = false, zfft = false;
  int Qz = 0, Wz = 0, kzq = 0;
  float* N3 = nullptr;     // [6][kxh][kyq][kzq]
  float* S3 = nullptr;     // [3][kxh][kyq][kzq]
  float2* Y3 = nullptr;    // [kxh][Qy][3 nz]
  float2* Z3H = nullptr;   // [3 nz][kxh][Qy]
  // reduced precision (every source through the split passes, z by the
  // direct sum): forward and demag-row inverse y DFT matrices
  DftMat yf, yiH;
  uint16_t* pkX = nullptr;  // x-transformed rows, split and packed for the forward DFT
  size_t pkX_bytes = 0;
  long long pkX_key = -1;
  uint16_t* pkH = nullptr;  // z-mixed demag planes, split and packed for the inverse DFT
  size_t pkH_bytes = 0;
  long long pkH_key = -1;
  // energy gradients (mm_backward_energy) as a source: work arrays and the S
  // spectra per z offset of the box
  float* adj_box = nullptr;
  float* adj_grid = nullptr;
  float2* adj_X = nullptr;
  float2* adj_Y = nullptr;
  float2* adj_Z = nullptr;
  float2* adj_YH = nullptr;
  float* adj_Sq = nullptr;
  size_t adj_bytes[7] = {};
  int adj_key[4] = {0, 0, 0, 0};  // dz_lo, planes, Qx, Qy of adj_Sq
  double adj_Ms = 0;
  Dir dir;   // hot path: coefficients around the other magnet
  Dir aux;   // mm_compute_potential output
  Dir cw;    // componentwise field variant: three coefficient boxes
  float2* cw_Y = nullptr;  // its y-forward spectra [3 nz][kxh][Qy]
  size_t cw_Y_bytes = 0;
  // eddy currents: the potential path on the magnet's own cells, the
  // rearranged input, E_sol, the Neumann source, phi_E, J, reduction scratch
  Dir eddy;
  float* ed_V = nullptr;
  float* ed_E = nullptr;
  double* ed_b = nullptr;
  double* ed_phi = nullptr;
  float* ed_J = nullptr;
  double* ed_part = nullptr;
  double* ed_stats = nullptr;  // max residual, max |b|, mean phi, mean b
  size_t ed_bytes[7] = {};
  // eddy currents coupled into the time step (a conducting magnet, sigma > 0):
  // B of the last accepted step, its rate, the eddy field used by the stages
  double sigma = 0;
  float* Bprev = nullptr;
  float* Bdot = nullptr;
  float* Heddy = nullptr;      // own eddy field plus the field of the other magnet's currents
  size_t eb_bytes[3] = {};
  bool B_valid = false, Heddy_valid = false;
  // as the source of the field of its currents inside the other magnet: the
  // potential path over the box around the other magnet, the three
  // rearranged-input coefficient boxes, and a scratch for the field
  Dir eddyx;
  float* ex_C3 = nullptr;
  float* ex_H = nullptr;
  size_t ex_bytes[2] = {};
};

struct TimedLaunch {
  int cls;
  cudaEvent_t a, b;
};

}  // namespace

struct mm_ctx {
  mm_options opt{};
  cudaStream_t st = nullptr;
  // the slider update of a step stage runs on `side` beside the LLG stage
  // launch; ev_fork / ev_join order it after the gather and before the next
  // reader of the state
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool mech_pending = false;
  std::string err;
  Magnet mag[2];
  std::map<int, FftRes> ffts;
  double Hext[3] = {0, 0, 0};
  // mechanics
  bool move = false;
  double mass = 0, k_spring = 0, v_drive = 0, gamma_v = 0, x0_spring = 0, e[3] = {1, 0, 0};
  double u_base[3] = {0, 0, 0};       // metres
  MechState host_mech{};
  MechState* mech = nullptr;          // device
  // pinned landing place of the readback that ends a step attempt; ev_done
  // marks its arrival, so a caller can queue other work behind it
  struct Readback {
    MechState mech;
    int err, pad;
  };
  Readback* rb = nullptr;
  cudaEvent_t ev_done = nullptr;
  int* err_flag = nullptr;            // device
  int* tickets = nullptr;             // device: last-block counters of the gather and stage launches
  bool k1_valid = false;
  long long accepted = 0, rejected = 0;
  // the most recent step attempts (oldest first), kAttemptLog at most
  struct Attempt {
    double t, dt, err;
    int accepted;
  };
  std::deque<Attempt> attempts;
  bool planned = false;
  // setup scratch (FP64 spectra generation)
  double2* gen_work = nullptr;
  size_t gen_work_bytes = 0;
  double* gen_q = nullptr;
  size_t gen_q_bytes = 0;
  double* W_dev = nullptr;
  size_t W_bytes = 0;
  // div / curl diagnostics: block sums, then the two totals
  double* dc_buf = nullptr;
  size_t dc_bytes = 0;
  // four-point difference variant: box coefficients, extended values
  float* fd4_C = nullptr;
  size_t fd4_C_bytes = 0;
  float* fd4_V = nullptr;
  size_t fd4_V_bytes = 0;
  // timing
  bool timing = false;
  std::vector<TimedLaunch> pending;
  std::vector<cudaEvent_t> free_events;
  double t_ms[kTimingClasses] = {};
  long long t_n[kTimingClasses] = {};
  long long launches = 0;
};

// eddy-current field of one magnet (steps 1-4 of Sec. III.B), defined with mm_eddy_field
static mm_status eddy_core(mm_ctx* ctx, int mag, const float* dBdt_dev, double sigma, float* H_dev, float* J_dev,
                           int* sweeps_out);
static mm_status cross_eddy_field(mm_ctx* ctx, int g, const float* J, float* H);

// ============================================================ helpers
namespace {

// A change made from outside the time step (m, displacement, slider, fields,
// materials, state) breaks the eddy fields' lag: B starts afresh.
void reset_eddy(mm_ctx* ctx) {
  for (auto& M : ctx->mag) M.B_valid = M.Heddy_valid = false;
}

mm_status fail(mm_ctx* c, mm_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? MM_ENOMEM : MM_ECUDA,            \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

#define CKS(expr)              \
  do {                         \
    mm_status s_ = (expr);     \
    if (s_ != MM_OK) return s_; \
  } while (0)

template <typename T>
mm_status ensure_buf(mm_ctx* ctx, T** p, size_t* have, size_t bytes) {
  if (*p && *have >= bytes) return MM_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (bytes == 0) return MM_OK;
  CK(cudaMalloc((void**)p, bytes));
  *have = bytes;
  return MM_OK;
}

mm_status alloc(mm_ctx* ctx, void** p, size_t bytes) {
  CK(cudaMalloc(p, bytes));
  return MM_OK;
}

int smooth_even_at_least(int n) {
  for (int q = std::max(2, n);; ++q) {
    if (q & 1) continue;
    int r = q;
    while (r % 2 == 0) r /= 2;
    while (r % 3 == 0) r /= 3;
    while (r % 5 == 0) r /= 5;
    if (r == 1) return q;
  }
}

// Fewest register-blocked stages whose radices (<= 16, as fft.cuh implements)
// multiply to L; largest radices first.
void radix_search(int L, int max_r, std::vector<int>& cur, std::vector<int>& best) {
  static const int kRadices[] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};
  if (L == 1) {
    if (best.empty() || cur.size() < best.size()) best = cur;
    return;
  }
  if (!best.empty() && cur.size() + 1 >= best.size()) return;
  for (int r : kRadices) {
    if (r > max_r || L % r) continue;
    cur.push_back(r);
    radix_search(L / r, r, cur, best);
    cur.pop_back();
  }
}

// Every ordering of every radix sequence with `stages` stages that multiplies to L.
void radix_orders(int L, int stages, std::vector<int>& cur, std::vector<std::vector<int>>& out) {
  static const int kRadices[] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};
  if ((int)cur.size() == stages) {
    if (L == 1) out.push_back(cur);
    return;
  }
  for (int r : kRadices) {
    if (L % r) continue;
    cur.push_back(r);
    radix_orders(L / r, stages, cur, out);
    cur.pop_back();
  }
}

// Shared-memory wavefronts of all stage loads of a plan (stores mirror them):
// the butterflies of fft_smem on 4 lines of stride L + 4, a warp's 32
// consecutive butterflies issuing one 8-byte access each, served per half
// warp with one wavefront per distinct 4-byte word in the busiest bank.
long long plan_wavefronts(int L, const std::vector<int>& radix) {
  const int nlines = 4, ldl = L + 4;
  long long total = 0;
  int Lb = L;
  std::vector<int> words;
  for (int R : radix) {
    const int M = Lb / R, per_line = L / R, nb = nlines * per_line;
    for (int k = 0; k < R; ++k)
      for (int w0 = 0; w0 < nb; w0 += 32)
        for (int h = w0; h < std::min(w0 + 32, nb); h += 16) {
          int count[32] = {0};
          words.clear();
          for (int b = h; b < std::min(h + 16, nb); ++b) {
            const int line = b / per_line, rem = b - line * per_line, blk = rem / M, n1 = rem - blk * M;
            const int a = line * ldl + blk * Lb + n1 + k * M;
            words.push_back(2 * a);
            words.push_back(2 * a + 1);
          }
          std::sort(words.begin(), words.end());
          words.erase(std::unique(words.begin(), words.end()), words.end());
          int worst = 0;
          for (int w : words) worst = std::max(worst, ++count[w & 31]);
          total += worst;
        }
    Lb /= R;
  }
  return total;
}

// The fewest stages; among those orderings, the ones within 5% of the fewest
// modelled shared-memory wavefronts (a stage whose blocks start in the same
// banks, e.g. an even radix last, costs up to several times the conflict-free
// count); of those the ones within the radix set the pass kernels are also
// built for (kRadixSetA), if any; then the largest last radix, the largest
// first radix, the fewest wavefronts.  The tie-breaks are measured: on GB300 the y pass
// of 540 = 4 9 15 ran 3% faster than 4 15 9 (model 598 vs 580 wavefronts), and
// the x passes of 2160 = 16 9 15 3% faster than 9 16 15 (2212 vs 2152).
std::vector<int> plan_radices(int L) {
  std::vector<int> cur, best;
  radix_search(L, 16, cur, best);
  if (best.empty()) return best;
  std::vector<std::vector<int>> orders;
  cur.clear();
  radix_orders(L, (int)best.size(), cur, orders);
  std::vector<long long> w(orders.size());
  long long wmin = plan_wavefronts(L, best);
  for (size_t i = 0; i < orders.size(); ++i) {
    w[i] = plan_wavefronts(L, orders[i]);
    wmin = std::min(wmin, w[i]);
  }
  auto in_a = [](const std::vector<int>& o) {
    for (int r : o)
      if (!(radix_bit(r) & kRadixSetA)) return false;
    return true;
  };
  bool any_a = false;
  for (size_t i = 0; i < orders.size(); ++i)
    if (20 * w[i] <= 21 * wmin && in_a(orders[i])) any_a = true;
  long long best_w = -1;
  for (size_t i = 0; i < orders.size(); ++i) {
    if (20 * w[i] > 21 * wmin || (any_a && !in_a(orders[i]))) continue;
    const auto& o = orders[i];
    const bool better = best_w < 0 || o.back() > best.back() ||
                        (o.back() == best.back() && (o.front() > best.front() ||
                                                     (o.front() == best.front() && w[i] < best_w)));
    if (better) {
      best = o;
      best_w = w[i];
    }
  }
  return best;
}

// ------------------------------------------------------------ autotuned plans
// Process-wide radix order per transform length, chosen by mm_autotune from
// timed runs of the pass kernels; the planner's model choice otherwise.
std::mutex g_tune_mu;
std::map<int, std::vector<int>> g_tuned;

bool tuned_plan(int L, std::vector<int>* out) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(L);
  if (it == g_tuned.end()) return false;
  if (out) *out = it->second;
  return true;
}

void set_tuned_plan(int L, const std::vector<int>& r) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned[L] = r;
}

// The candidates an autotuner times for length L: the model's choice first,
// then the other orderings of the fewest-stage factorisations by modelled
// shared-memory wavefronts, at most `k` in all.
std::vector<std::vector<int>> plan_candidates(int L, int k) {
  std::vector<std::vector<int>> out;
  const std::vector<int> model = plan_radices(L);
  if (model.empty()) return out;
  out.push_back(model);
  std::vector<int> cur;
  std::vector<std::vector<int>> orders;
  radix_orders(L, (int)model.size(), cur, orders);
  std::vector<std::pair<long long, std::vector<int>>> w;
  for (const auto& o : orders) w.push_back({plan_wavefronts(L, o), o});
  std::sort(w.begin(), w.end());
  for (const auto& e : w) {
    if ((int)out.size() >= k) break;
    if (std::find(out.begin(), out.end(), e.second) == out.end()) out.push_back(e.second);
  }
  return out;
}

// FFT resources of length L (plan, twiddle and position tables), cached per
// context; the plan is the autotuned one when mm_autotune has chosen it.
mm_status get_fft(mm_ctx* ctx, int L, FftTables* out) {
  const int key = L;
  auto it = ctx->ffts.find(key);
  if (it != ctx->ffts.end()) {
    *out = it->second.t;
    return MM_OK;
  }
  FftRes R;
  int p2 = 0, p3 = 0, p5 = 0, r = L;
  while (r % 2 == 0) { r /= 2; ++p2; }
  while (r % 3 == 0) { r /= 3; ++p3; }
  while (r % 5 == 0) { r /= 5; ++p5; }
  if (r != 1) return fail(ctx, MM_EINVAL, "FFT length is not 2^a 3^b 5^c");
  (void)p2; (void)p3; (void)p5;
  std::vector<int> radix;
  if (!tuned_plan(L, &radix)) radix = plan_radices(L);
  if (radix.empty() || (int)radix.size() > kMaxStages)
    return fail(ctx, MM_ENOTSUP, "FFT length has too many factors");
  FftPlanDev P{};
  P.L = L;
  P.nstages = (int)radix.size();
  int Lb = L;
  for (int s = 0; s < P.nstages; ++s) {
    P.radix[s] = radix[s];
    P.blocklen[s] = Lb;
    const unsigned per_line = (unsigned)(L / radix[s]);
    const unsigned M = (unsigned)(Lb / radix[s]);
    // 0 marks a divisor of 1 (the quotient is the dividend)
    P.magic_per_line[s] = per_line == 1 ? 0u : (unsigned)(0xFFFFFFFFull / per_line) + 1u;
    P.magic_M[s] = M == 1 ? 0u : (unsigned)(0xFFFFFFFFull / M) + 1u;
    P.magic_r[s] = (unsigned)(0xFFFFFFFFull / (unsigned)radix[s]) + 1u;
    Lb /= radix[s];
  }
  // stage twiddle tables: W_Lb^{n1 k} at (k - 1) M + n1, k = 1 .. R-1, n1 < M = Lb / R
  std::vector<float2> twf;
  std::vector<double2> twd;
  for (int s = 0; s < P.nstages; ++s) {
    const int R = P.radix[s], Lbs = P.blocklen[s], M = Lbs / R;
    P.stw_off[s] = (int)twf.size();
    for (int k = 1; k < R; ++k)
      for (int n1 = 0; n1 < M; ++n1) {
        const long long t = ((long long)n1 * k) % Lbs;
        const double ang = -2.0 * 3.14159265358979323846 * (double)t / (double)Lbs;
        twd.push_back(make_double2(cos(ang), sin(ang)));
        twf.push_back(make_float2((float)twd.back().x, (float)twd.back().y));
      }
  }
  if (twf.empty()) {  // a single-stage plan reads no table
    twf.push_back(make_float2(1.f, 0.f));
    twd.push_back(make_double2(1.0, 0.0));
  }
  const size_t ntw = twf.size();
  std::vector<int> pos(L), freq(L);
  for (int k = 0; k < L; ++k) {
    int p = 0, rem = k, B = L;
    for (int s = 0; s < P.nstages; ++s) {
      const int M = B / P.radix[s];
      p += M * (rem % P.radix[s]);
      rem /= P.radix[s];
      B = M;
    }
    pos[k] = p;
    freq[p] = k;
  }
  CKS(alloc(ctx, (void**)&R.tw_f, sizeof(float2) * ntw));
  CKS(alloc(ctx, (void**)&R.tw_d, sizeof(double2) * ntw));
  CKS(alloc(ctx, (void**)&R.pos, sizeof(int) * L));
  CKS(alloc(ctx, (void**)&R.freq, sizeof(int) * L));
  CK(cudaMemcpy(R.tw_f, twf.data(), sizeof(float2) * ntw, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(R.tw_d, twd.data(), sizeof(double2) * ntw, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(R.pos, pos.data(), sizeof(int) * L, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(R.freq, freq.data(), sizeof(int) * L, cudaMemcpyHostToDevice));
  R.t.plan = P;
  R.t.tw_f = R.tw_f;
  R.t.tw_d = R.tw_d;
  R.t.pos = R.pos;
  R.t.freq = R.freq;
  ctx->ffts[key] = R;
  *out = R.t;
  return MM_OK;
}

double u_cells(const mm_ctx* ctx, int a, double x) {
  return (ctx->u_base[a] + x * ctx->e[a]) / ctx->mag[0].d[a];
}

// ------------------------------------------------------------ timing
cudaEvent_t grab_event(mm_ctx* ctx) {
  if (!ctx->free_events.empty()) {
    cudaEvent_t e = ctx->free_events.back();
    ctx->free_events.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

struct Timer {
  mm_ctx* ctx;
  int cls;
  cudaEvent_t a = nullptr, b = nullptr;
  Timer(mm_ctx* c, int k) : ctx(c), cls(k) {
    ctx->launches++;
    if (ctx->timing) {
      a = grab_event(ctx);
      b = grab_event(ctx);
      cudaEventRecord(a, ctx->st);
    }
  }
  ~Timer() {
    if (a) {
      cudaEventRecord(b, ctx->st);
      ctx->pending.push_back({cls, a, b});
    }
  }
};

void drain_timing(mm_ctx* ctx) {
  if (ctx->pending.empty()) return;
  cudaStreamSynchronize(ctx->st);
  for (auto& p : ctx->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    ctx->t_ms[p.cls] += ms;
    ctx->t_n[p.cls] += 1;
    ctx->free_events.push_back(p.a);
    ctx->free_events.push_back(p.b);
  }
  ctx->pending.clear();
}

// ------------------------------------------------------------ planning
// B-spline prefilter taps sqrt(3) z1^|i|, z1 = sqrt(3) - 2
void fir_taps(double* h) {
  const double z1 = sqrt(3.0) - 2.0;
  for (int i = 0; i <= kFirHalf; ++i) h[i] = sqrt(3.0) * pow(z1, i);
}

int host_mirror(int j, int b) {
  if (b <= 1) return 0;
  const int P = 2 * b - 2;
  j %= P;
  if (j < 0) j += P;
  return j < b ? j : P - j;
}

// x (a = 0) or y (a = 1) periodic (mm_options.periodic); z never
bool periodic_axis(const mm_ctx* ctx, int a) {
  return a < 2 && (ctx->opt.periodic & (1 << a)) != 0;
}

KernelPlan kernel_plan(const mm_ctx* ctx, const Magnet& S) {
  KernelPlan K{S.Qx, S.Qy, S.Wx, S.Wy, S.nz};
  K.px = periodic_axis(ctx, 0) ? 1 : 0;
  K.py = periodic_axis(ctx, 1) ? 1 : 0;
  K.R = ctx->opt.pbc_images;
  return K;
}

void dir_geometry(const mm_ctx* ctx, int s, bool full_box, Dir* D) {
  const int t = 1 - s;
  const Magnet& S = ctx->mag[s];
  const Magnet& T = ctx->mag[t];
  const double sigma = t == 1 ? 1.0 : -1.0;
  const int nt[3] = {T.nx, T.ny, T.nz};
  const int m = ctx->opt.margin;
  for (int a = 0; a < 3; ++a) {
    const double su = sigma * u_cells(ctx, a, ctx->host_mech.x);
    const int U = (int)floor(su);
    D->U0[a] = U;
    if (periodic_axis(ctx, a)) {
      // the potential lives on every node of the period (Sec. III.A: the
      // margin beyond the domain is the other side's values)
      const int P = a == 0 ? S.nx : S.ny;
      D->box_lo[a] = 0;
      D->box_len[a] = P;
      D->guard[a] = 0;
      D->start[a] = 0;
      D->r[a] = P;
      continue;
    }
    const long long Dd = T.off[a] - S.off[a];
    D->box_lo[a] = (int)(Dd + U - 1 - m);
    D->box_len[a] = nt[a] + 3 + 2 * m;
    const int g = (!full_box && ctx->move && ctx->e[a] != 0.0) ? 1 : 0;
    D->guard[a] = g;
    if (full_box) {
      D->start[a] = 0;
      D->r[a] = D->box_len[a];
    } else {
      D->start[a] = m - g;
      D->r[a] = nt[a] + 3 + 2 * g;
    }
  }
  D->full_box = full_box;
}

int window_needed(const Magnet& S, const Dir& D, int a) {
  const int n = a == 0 ? S.nx : (a == 1 ? S.ny : S.nz);
  int w = n - 1;  // self-demag offsets
  w = std::max(w, std::abs(D.box_lo[a] - (n - 1)));
  w = std::max(w, std::abs(D.box_lo[a] + D.box_len[a] - 1));
  return w;
}

// kind 0: the W-folded S spectra of the potential (Tq [n_out][nz][3]);
// kind 1: the W-folded rows of -N of the componentwise field variant
// (Tq [3][n_out][nz][3]).
mm_status build_T(mm_ctx* ctx, int s, Dir* D, int kind = 0) {
  Magnet& S = ctx->mag[s];
  const int n_out = D->r[2];
  const int bz = D->box_len[2];
  if (D->Tq && D->Tq_box_lo_z == D->box_lo[2] && D->Tq_bz == bz && D->Tq_start_z == D->start[2] &&
      D->Tq_nout == n_out && D->Tq_prefilter == D->prefilter && D->Tq_Q[0] == S.Qx &&
      D->Tq_Q[1] == S.Qy && D->Tq_kind == kind)
    return MM_OK;
  FftTables fx, fy;
  CKS(get_fft(ctx, S.Qx, &fx));
  CKS(get_fft(ctx, S.Qy, &fy));
  const size_t qsize = (size_t)S.kxh * S.kyq;
  CKS(ensure_buf(ctx, &D->Tq, &D->Tq_bytes, sizeof(float) * (size_t)(kind ? 3 : 1) * n_out * S.nz * 3 * qsize));
  // z mixing matrix: rows = output planes, columns = box planes
  std::vector<double> W((size_t)n_out * bz, 0.0);
  double h[kFirHalf + 1];
  fir_taps(h);
  for (int o = 0; o < n_out; ++o) {
    const int c = D->start[2] + o;
    if (D->prefilter) {
      for (int i = -kFirHalf; i <= kFirHalf; ++i) W[(size_t)o * bz + host_mirror(c - i, bz)] += h[std::abs(i)];
    } else {
      W[(size_t)o * bz + c] = 1.0;
    }
  }
  CKS(ensure_buf(ctx, &ctx->W_dev, &ctx->W_bytes, sizeof(double) * W.size()));
  CK(cudaMemcpyAsync(ctx->W_dev, W.data(), sizeof(double) * W.size(), cudaMemcpyHostToDevice, ctx->st));
  const size_t plane = (size_t)S.Qx * S.Qy;
  CKS(ensure_buf(ctx, &ctx->gen_work, &ctx->gen_work_bytes, sizeof(double2) * 2 * 6 * plane));
  const int nplanes = bz + S.nz - 1;
  CKS(ensure_buf(ctx, &ctx->gen_q, &ctx->gen_q_bytes, sizeof(double) * (size_t)nplanes * (kind ? 6 : 3) * qsize));
  const KernelPlan K = kernel_plan(ctx, S);
  const double scale = S.Ms / ((double)S.Qx * S.Qy);
  if (kind == 0)
    CK(build_T_spectra(K, fx, fy, S.d[0], S.d[1], S.d[2], scale, D->box_lo[2], bz, n_out, ctx->W_dev, D->Tq,
                       ctx->gen_work, ctx->gen_q, ctx->st));
  else  // H = -N M
    CK(build_TN_spectra(K, fx, fy, S.d[0], S.d[1], S.d[2], -scale, D->box_lo[2], bz, n_out, ctx->W_dev, D->Tq,
                        ctx->gen_work, ctx->gen_q, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));  // W_dev / scratch reuse
  D->Tq_box_lo_z = D->box_lo[2];
  D->Tq_bz = bz;
  D->Tq_start_z = D->start[2];
  D->Tq_nout = n_out;
  D->Tq_prefilter = D->prefilter;
  D->Tq_Q[0] = S.Qx;
  D->Tq_Q[1] = S.Qy;
  D->Tq_kind = kind;
  return MM_OK;
}

mm_status alloc_dir_outputs(mm_ctx* ctx, int s, Dir* D) {
  Magnet& S = ctx->mag[s];
  const Magnet& T = ctx->mag[1 - s];
  CKS(ensure_buf(ctx, &D->YC, &D->YC_bytes, sizeof(float2) * (size_t)D->r[2] * S.kxh * D->r[1]));
  CKS(ensure_buf(ctx, &D->C, &D->C_bytes, sizeof(float) * (size_t)D->r[2] * D->r[1] * D->r[0]));
  D->ntiles = gather_tiles(T.nx, T.ny, T.nz);
  CKS(ensure_buf(ctx, &D->partial, &D->partial_bytes, sizeof(float2) * 4 * (size_t)D->ntiles));
  if (S.thick)
    CKS(ensure_buf(ctx, &D->Z3C, &D->Z3C_bytes, sizeof(float2) * (size_t)D->r[2] * S.kxh * S.Qy));
  return MM_OK;
}

mm_status alloc_magnet(mm_ctx* ctx, Magnet& M) {
  if (M.m) return MM_OK;
  const size_t b = sizeof(float) * 3 * M.N;
  CKS(alloc(ctx, (void**)&M.m, b));
  CK(cudaMemset(M.m, 0, b));
  for (int i = 0; i < 2; ++i) CKS(alloc(ctx, (void**)&M.ys[i], b));
  for (int i = 0; i < 7; ++i) CKS(alloc(ctx, (void**)&M.k[i], b));
  CKS(alloc(ctx, (void**)&M.Hself, b));
  CKS(alloc(ctx, (void**)&M.Hstray, b));
  CKS(alloc(ctx, (void**)&M.scratch3, b));
  M.nerr = (int)((M.N + 255) / 256);
  CKS(alloc(ctx, (void**)&M.err_partial, sizeof(float) * M.nerr));
  return MM_OK;
}

// FP64 generation of the 3D N and S spectra of a thick source (one-time set-up).
mm_status build_spectra_3d_all(mm_ctx* ctx, Magnet& S, const FftTables& fx, const FftTables& fy) {
  FftTables fz;
  CKS(get_fft(ctx, S.Qz, &fz));
  const size_t qsize = (size_t)S.kxh * S.kyq;
  double* q2 = nullptr;
  double* qtmp = nullptr;
  double2* zl = nullptr;
  CKS(alloc(ctx, (void**)&q2, sizeof(double) * 6 * (size_t)S.Qz * qsize));
  mm_status st = alloc(ctx, (void**)&qtmp, sizeof(double) * 6 * qsize);
  if (st == MM_OK) st = alloc(ctx, (void**)&zl, sizeof(double2) * qsize * S.Qz);
  if (st == MM_OK) {
    const KernelPlan3 K{S.Qx, S.Qy, S.Qz, S.Wx, S.Wy, S.Wz};
    const double norm = (double)S.Qx * S.Qy * S.Qz;
    cudaError_t e = build_spectra_3d(1, K, fx, fy, fz, S.d[0], S.d[1], S.d[2], -S.Ms / norm, S.N3,
                                     ctx->gen_work, q2, qtmp, zl, ctx->st);
    if (e == cudaSuccess)
      e = build_spectra_3d(0, K, fx, fy, fz, S.d[0], S.d[1], S.d[2], S.Ms / norm, S.S3, ctx->gen_work, q2,
                           qtmp, zl, ctx->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    if (e != cudaSuccess) st = fail(ctx, MM_ECUDA, std::string("3D spectra: ") + cudaGetErrorString(e));
  }
  cudaFree(q2); cudaFree(qtmp); cudaFree(zl);
  return st;
}

// (Re)plan both sources for the current displacement; rebuild spectra as needed.
mm_status ensure_plan(mm_ctx* ctx) {
  for (int g = 0; g < 2; ++g) {
    if (!ctx->mag[g].grid) return fail(ctx, MM_EINVAL, "grid of magnet " + std::to_string(g) + " not set");
    if (!ctx->mag[g].mat) return fail(ctx, MM_EINVAL, "material of magnet " + std::to_string(g) + " not set");
  }
  for (int a = 0; a < 2; ++a) {
    if (!periodic_axis(ctx, a)) continue;
    const int n0 = a == 0 ? ctx->mag[0].nx : ctx->mag[0].ny;
    const int n1 = a == 0 ? ctx->mag[1].nx : ctx->mag[1].ny;
    if (n0 != n1)
      return fail(ctx, MM_EINVAL, "periodic boundaries: both magnets must span the period (equal nx / ny)");
    if (n0 % 2 || smooth_even_at_least(n0) != n0)
      return fail(ctx, MM_ENOTSUP, "periodic boundaries: the period must be even and 2^a 3^b 5^c cells");
  }
  for (int s = 0; s < 2; ++s) {
    Magnet& S = ctx->mag[s];
    Dir& D = S.dir;
    dir_geometry(ctx, s, false, &D);
    D.prefilter = 1;
    // separate y / z passes when the source is thick or the box around the
    // target is tall; z by FFT only for sources thicker than kMaxNzDirect
    // (the reduced-precision form takes every source through the separate
    // passes: its y transforms are the tensor-core DFT products)
    const bool mixed = ctx->opt.precision == MM_MIXED;
    const bool thick = S.nz > kMaxNz || ctx->mag[1 - s].nz > kMaxNz || mixed;
    const bool zfft = thick && S.nz > kMaxNzDirect;
    if (zfft && mixed)
      return fail(ctx, MM_ENOTSUP, "reduced precision: sources of more than 8 layers (z by FFT)");
    if (zfft && ctx->opt.periodic)
      return fail(ctx, MM_ENOTSUP, "periodic boundaries: sources of more than 8 layers");
    const bool px = periodic_axis(ctx, 0), py = periodic_axis(ctx, 1);
    const int wx = window_needed(S, D, 0), wy = window_needed(S, D, 1), wz = window_needed(S, D, 2);
    // a periodic axis: the circular grid is the period itself
    const bool regrid = S.Qx == 0 || (px ? S.Qx != S.nx : 2 * wx + 2 > S.Qx) ||
                        (py ? S.Qy != S.ny : 2 * wy + 2 > S.Qy) || thick != S.thick ||
                        zfft != S.zfft || (zfft && 2 * wz + 2 > S.Qz);
    if (regrid) {
      S.thick = thick;
      S.zfft = zfft;
      S.Wx = wx + kWindowSlack;
      S.Wy = wy + kWindowSlack;
      S.Qx = px ? S.nx : smooth_even_at_least(2 * S.Wx + 2);
      S.Qy = py ? S.ny : smooth_even_at_least(2 * S.Wy + 2);
      // keep the window inside the grid: the largest W with 2W + 2 <= Q
      // (periodic axes ignore it: every offset of the period counts)
      S.Wx = (S.Qx - 2) / 2;
      S.Wy = (S.Qy - 2) / 2;
      S.kxh = S.Qx / 2 + 1;
      S.kyq = S.Qy / 2 + 1;
      if (zfft) {
        S.Wz = wz + kWindowSlack;
        S.Qz = smooth_even_at_least(2 * S.Wz + 2);
        S.Wz = (S.Qz - 2) / 2;
        S.kzq = S.Qz / 2 + 1;
      } else {
        S.Qz = S.Wz = S.kzq = 0;
      }
      if ((size_t)(kRowsPerCta / 2) * S.Qx * sizeof(float2) > 220 * 1024)
        return fail(ctx, MM_ENOTSUP, "x extent too large for one shared-memory line");
      if (!thick) {
        const int P = std::max(3 * S.nz, 3 * S.nz + D.r[2]);
        if ((size_t)P * S.Qy * sizeof(float2) > 220 * 1024)
          return fail(ctx, MM_ENOTSUP, "y extent x planes too large for the fused y pass");
      } else {
        if ((size_t)(S.Qy + 1) * sizeof(float2) + 4096 > 220 * 1024)
          return fail(ctx, MM_ENOTSUP, "y extent too large for one shared-memory line");
        if (zfft && (size_t)4 * zpass_tile(S.Qz) * (S.Qz + 1) * sizeof(float2) + 8192 > 220 * 1024)
          return fail(ctx, MM_ENOTSUP, "z extent too large for the z pass");
      }
      S.Nq_Ms = 0;  // force a spectra rebuild
      cudaFree(S.X1); cudaFree(S.YH); cudaFree(S.Nq);
      cudaFree(S.N3); cudaFree(S.S3); cudaFree(S.Y3); cudaFree(S.Z3H);
      S.X1 = S.YH = S.Y3 = S.Z3H = nullptr;
      S.Nq = S.N3 = S.S3 = nullptr;
      S.aux.valid = false;
    }
    const size_t qsize = (size_t)S.kxh * S.kyq;
    if (!S.X1) {
      CKS(alloc(ctx, (void**)&S.X1, sizeof(float2) * 3 * S.nz * S.kxh * (size_t)S.ny));
      CKS(alloc(ctx, (void**)&S.YH, sizeof(float2) * 3 * S.nz * S.kxh * (size_t)S.ny));
      if (!S.zfft) {
        CKS(alloc(ctx, (void**)&S.Nq, sizeof(float) * 6 * S.nz * qsize));
      } else {
        CKS(alloc(ctx, (void**)&S.N3, sizeof(float) * 6 * qsize * S.kzq));
        CKS(alloc(ctx, (void**)&S.S3, sizeof(float) * 3 * qsize * S.kzq));
      }
      if (S.thick) {
        CKS(alloc(ctx, (void**)&S.Y3, sizeof(float2) * (size_t)S.kxh * S.Qy * 3 * S.nz));
        CKS(alloc(ctx, (void**)&S.Z3H, sizeof(float2) * (size_t)3 * S.nz * S.kxh * S.Qy));
      }
    }
    if (S.Nq_Ms != S.Ms) {
      FftTables fx, fy;
      CKS(get_fft(ctx, S.Qx, &fx));
      CKS(get_fft(ctx, S.Qy, &fy));
      const size_t plane = (size_t)S.Qx * S.Qy;
      CKS(ensure_buf(ctx, &ctx->gen_work, &ctx->gen_work_bytes, sizeof(double2) * 2 * 6 * plane));
      if (!S.zfft) {
        CKS(ensure_buf(ctx, &ctx->gen_q, &ctx->gen_q_bytes,
                       std::max(ctx->gen_q_bytes, sizeof(double) * 6 * qsize)));
        const KernelPlan K = kernel_plan(ctx, S);
        CK(build_N_spectra(K, fx, fy, S.d[0], S.d[1], S.d[2], -S.Ms / ((double)S.Qx * S.Qy), S.Nq,
                           ctx->gen_work, ctx->gen_q, ctx->st));
      } else {
        CKS(build_spectra_3d_all(ctx, S, fx, fy));
      }
      CK(cudaStreamSynchronize(ctx->st));
      S.Nq_Ms = S.Ms;
    }
    if (!S.zfft) CKS(build_T(ctx, s, &D));
    CKS(alloc_dir_outputs(ctx, s, &D));
    D.valid = true;
  }
  ctx->planned = true;
  return MM_OK;
}

// Re-plan when the whole-cell part of the displacement moved outside the guard.
mm_status replan_if_needed(mm_ctx* ctx) {
  if (!ctx->planned) return ensure_plan(ctx);
  for (int s = 0; s < 2; ++s) {
    const Dir& D = ctx->mag[s].dir;
    const double sigma = s == 0 ? 1.0 : -1.0;
    for (int a = 0; a < 3; ++a) {
      if (periodic_axis(ctx, a)) continue;  // the box is the whole period
      const int U = (int)floor(sigma * u_cells(ctx, a, ctx->host_mech.x));
      if (U != D.U0[a]) return ensure_plan(ctx);
    }
  }
  return MM_OK;
}

// The context stream waits for a slider update still running on the side stream.
mm_status join_mech(mm_ctx* ctx) {
  if (!ctx->mech_pending) return MM_OK;
  CK(cudaStreamWaitEvent(ctx->st, ctx->ev_join, 0));
  ctx->mech_pending = false;
  return MM_OK;
}

mm_status upload_mech(mm_ctx* ctx) {
  CKS(join_mech(ctx));
  MechState& H = ctx->host_mech;
  H.xs = H.x; H.vs = H.v; H.ts = H.t;
  for (int a = 0; a < 3; ++a) H.u[a] = u_cells(ctx, a, H.x);
  split_displacement(H.u, H.ucell, H.ufrac);
  CK(cudaMemcpyAsync(ctx->mech, &H, sizeof(MechState), cudaMemcpyHostToDevice, ctx->st));
  return MM_OK;
}

// ------------------------------------------------------------ launch sequences
Launch<XFwdJob> xfwd_launch(mm_ctx* ctx, const float* in[2], const int* which, int n, int* Qmax) {
  Launch<XFwdJob> L{};
  L.njobs = n;
  int tiles = 0;
  *Qmax = 0;
  for (int i = 0; i < n; ++i) {
    Magnet& S = ctx->mag[which[i]];
    XFwdJob& J = L.job[i];
    J.m = in[which[i]];
    J.out = S.X1;
    J.nx = S.nx; J.ny = S.ny; J.nz = S.nz; J.kxh = S.kxh;
    get_fft(ctx, S.Qx, &J.fx);
    L.tile_start[i] = tiles;
    tiles += (3 * S.nz * S.ny + kRowsPerCta - 1) / kRowsPerCta;
    *Qmax = std::max(*Qmax, S.Qx);
  }
  L.tile_start[n] = tiles;
  return L;
}

// The packed matrix of `spec` in *M, rebuilt (FP64 entries, on the stream)
// when the geometry it was built for has changed.
static mm_status ensure_dft(mm_ctx* ctx, DftMat* M, const DftSpec& spec) {
  if (M->valid && memcmp(&M->spec, &spec, sizeof spec) == 0) return MM_OK;
  const DftShape sh = dft_shape(spec.Nc, spec.Kc);
  const size_t bytes = dft_matrix_elems(sh) * sizeof(uint16_t);
  M->valid = false;
  CKS(ensure_buf(ctx, &M->hi, &M->hi_bytes, bytes));
  CKS(ensure_buf(ctx, &M->lo, &M->lo_bytes, bytes));
  CK(launch_dft_pack(spec, sh, M->hi, M->lo, ctx->st));
  M->spec = spec;
  M->shape = sh;
  M->valid = true;
  return MM_OK;
}

static DftJob dft_job(mm_ctx* ctx, const DftMat& M, const float2* A, int lda, int rows, float2* D, int ldd) {
  DftJob J{};
  J.A = A; J.lda = lda; J.rows = rows; J.Kc = M.spec.Kc;
  J.Bhi = M.hi; J.Blo = M.lo;
  J.ntile = M.shape.ntile; J.ntiles = M.shape.ntiles; J.kchunks = M.shape.kchunks; J.Nc = M.spec.Nc;
  J.D = D; J.ldd = ldd;
  J.err = ctx->err_flag;
  return J;
}

// A packed split operand of `rows` rows and Kc complex columns: allocated,
// and zeroed whenever its layout changes (the K padding of the last chunk is
// never written and must read as zero: the matrix is zero there, and a stale
// NaN would not cancel)
static mm_status ensure_packed(mm_ctx* ctx, uint16_t** p, size_t* have, long long* key, int rows, int Kc) {
  DftShape sh = dft_shape(1, Kc);
  const size_t bytes = dft_a_bytes(rows, sh);
  const long long k = (long long)rows * 1000003LL + Kc;
  if (*p && *have >= bytes && *key == k) return MM_OK;
  CKS(ensure_buf(ctx, p, have, bytes));
  CK(cudaMemsetAsync(*p, 0, bytes, ctx->st));
  *key = k;
  return MM_OK;
}

// what: bit 1 = own demag, bit 2 = coefficients of Dir (hot or aux)
mm_status run_source_passes(mm_ctx* ctx, const float* in[2], const int* which, int n, const int* what,
                            Dir* const* dirs) {
  cudaStream_t st = ctx->st;
  int Qmax = 0;
  {
    Launch<XFwdJob> L = xfwd_launch(ctx, in, which, n, &Qmax);
    if (ctx->opt.precision == MM_MIXED)  // the forward y DFT's split operand, written by this pass
      for (int i = 0; i < n; ++i) {
        Magnet& S = ctx->mag[which[i]];
        CKS(ensure_packed(ctx, &S.pkX, &S.pkX_bytes, &S.pkX_key, 3 * S.nz * S.kxh, S.ny));
        L.job[i].pk = S.pkX;
      }
    Timer t(ctx, 0);
    CK(launch_xfwd(L, Qmax, st));
  }
  // y stage: thin sources in the fused y pass (z by plane mixing); thick
  // sources through y forward, z pass and y inverse (z by FFT)
  {
    Launch<YJob> L{};
    int tiles = 0, nj = 0;
    size_t smem = 0;
    for (int i = 0; i < n; ++i) {
      Magnet& S = ctx->mag[which[i]];
      if (S.thick) continue;
      Dir* D = dirs[i];
      YJob& J = L.job[nj];
      J.in = S.X1;
      J.nz = S.nz; J.ny = S.ny; J.kxh = S.kxh; J.kyq = S.kyq;
      CKS(get_fft(ctx, S.Qy, &J.fy));
      J.do_H = (what[i] & 1) ? 1 : 0;
      J.Nq = S.Nq;
      J.outH = S.YH;
      J.do_C = (what[i] & 2) ? 1 : 0;
      if (J.do_C) {
        J.n_out = D->r[2];
        J.Tq = D->Tq;
        J.outC = D->YC;
        J.box_lo = D->box_lo[1];
        J.box_len = D->box_len[1];
        J.start = D->start[1];
        J.r = D->r[1];
        J.fir = D->prefilter;
        J.periodic = periodic_axis(ctx, 1) ? 1 : 0;
      }
      const int Pout = (J.do_H ? 3 * S.nz : 0) + (J.do_C ? J.n_out : 0);
      const int P = std::max(3 * S.nz, Pout);
      // spectra columns + the prefilter index table
      smem = std::max(smem, (size_t)P * S.Qy * sizeof(float2) + ypass_table_bytes(J.do_C ? J.r : 0));
      L.tile_start[nj] = tiles;
      tiles += S.kxh;
      ++nj;
    }
    if (nj) {
      L.njobs = nj;
      L.tile_start[nj] = tiles;
      Timer t(ctx, 1);
      CK(launch_ypass(L, smem, st));
    }
  }
  {
    Launch<YFwdJob> Lf{};
    Launch<ZJob> Lz{};
    Launch<ZMixJob> Lm{};
    Launch<YInvJob> Li{};
    // reduced precision: the y transforms as tensor-core DFT products
    Launch<DftJob> Ldf{}, Ldi{};
    const bool mixed = ctx->opt.precision == MM_MIXED;
    int nf = 0, tf = 0, nzj = 0, tz = 0, nm = 0, tm = 0, ni = 0, ti = 0;
    int ndf = 0, tdf = 0, ndi = 0, tdi = 0;
    for (int i = 0; i < n; ++i) {
      Magnet& S = ctx->mag[which[i]];
      if (!S.thick) continue;
      Dir* D = dirs[i];
      const bool do_H = (what[i] & 1) != 0, do_C = (what[i] & 2) != 0;
      FftTables fy;
      CKS(get_fft(ctx, S.Qy, &fy));
      // planes per y-pass CTA: about 48 KB of lines, at most 16
      const int group = std::max(1, std::min(16, (int)((48 * 1024) / ((S.Qy + 1) * sizeof(float2)))));
      const int P3 = 3 * S.nz;
      const int natural = S.zfft ? 0 : 1;
      if (mixed) {
        DftSpec f{};
        f.kind = kDftForward; f.Q = S.Qy; f.Nc = S.Qy; f.Kc = S.ny;
        CKS(ensure_dft(ctx, &S.yf, f));
        Ldf.job[ndf] = dft_job(ctx, S.yf, S.X1, S.ny, P3 * S.kxh, S.Y3, S.Qy);
        Ldf.job[ndf].Apk = S.pkX;  // written by the x-forward pass
        Ldf.tile_start[ndf] = tdf;
        tdf += dft_tiles(P3 * S.kxh, S.yf.shape);
        ++ndf;
      } else {
        YFwdJob& F = Lf.job[nf];
        F.in = S.X1; F.out = S.Y3; F.planes = P3; F.ny = S.ny; F.kxh = S.kxh; F.group = group; F.fy = fy;
        F.natural = natural;
        Lf.tile_start[nf] = tf;
        tf += S.kxh * ((P3 + group - 1) / group);
        ++nf;
      }
      if (S.zfft) {
        FftTables fz;
        CKS(get_fft(ctx, S.Qz, &fz));
        ZJob& Z = Lz.job[nzj];
        Z.in = S.Y3; Z.nz = S.nz; Z.kxh = S.kxh; Z.fy = fy; Z.fz = fz; Z.kyq = S.kyq; Z.kzq = S.kzq;
        Z.N3 = S.N3; Z.S3 = S.S3;
        Z.do_H = do_H ? 1 : 0;
        Z.do_C = do_C ? 1 : 0;
        Z.outH = S.Z3H;
        if (do_C) {
          Z.outC = D->Z3C;
          Z.box_lo = D->box_lo[2]; Z.box_len = D->box_len[2]; Z.start = D->start[2]; Z.r = D->r[2];
          Z.fir = D->prefilter;
        }
        Z.ztile = zpass_tile(S.Qz);
        Lz.tile_start[nzj] = tz;
        tz += S.kxh * zpass_tiles(S.Qy, Z.ztile);
        ++nzj;
      } else {
        ZMixJob& M = Lm.job[nm];
        M.in = S.Y3; M.nz = S.nz; M.kxh = S.kxh; M.Qy = S.Qy; M.kyq = S.kyq;
        M.Nq = S.Nq; M.Tq = do_C ? D->Tq : nullptr;
        M.nH = do_H ? P3 : 0;
        M.n_out = do_C ? D->r[2] : 0;
        M.outH = S.Z3H;
        M.outC = do_C ? D->Z3C : nullptr;
        Lm.tile_start[nm] = tm;
        tm += S.kxh * zmix_tiles(S.kyq, M.nH + M.n_out);
        ++nm;
      }
      if (mixed) {
        if (do_H) {
          DftSpec h{};
          h.kind = kDftInverse; h.Q = S.Qy; h.Nc = S.ny; h.Kc = S.Qy;
          CKS(ensure_dft(ctx, &S.yiH, h));
          // the mixing pass writes the split operand itself
          CKS(ensure_packed(ctx, &S.pkH, &S.pkH_bytes, &S.pkH_key, P3 * S.kxh, S.Qy));
          Lm.job[nm - 1].pkH = S.pkH;
          Ldi.job[ndi] = dft_job(ctx, S.yiH, S.Z3H, S.Qy, P3 * S.kxh, S.YH, S.ny);
          Ldi.job[ndi].Apk = S.pkH;
          Ldi.tile_start[ndi] = tdi;
          tdi += dft_tiles(P3 * S.kxh, S.yiH.shape);
          ++ndi;
        }
        if (do_C) {
          DftSpec c{};
          c.kind = kDftInversePrefilter; c.Q = S.Qy; c.Nc = D->r[1]; c.Kc = S.Qy;
          c.box_lo = D->box_lo[1]; c.box_len = D->box_len[1]; c.start = D->start[1];
          c.periodic = periodic_axis(ctx, 1) ? 1 : 0;
          c.fir = D->prefilter;
          CKS(ensure_dft(ctx, &D->yiC, c));
          CKS(ensure_packed(ctx, &D->pkC, &D->pkC_bytes, &D->pkC_key, D->r[2] * S.kxh, S.Qy));
          Lm.job[nm - 1].pkC = D->pkC;
          Ldi.job[ndi] = dft_job(ctx, D->yiC, D->Z3C, S.Qy, D->r[2] * S.kxh, D->YC, D->r[1]);
          Ldi.job[ndi].Apk = D->pkC;
          Ldi.tile_start[ndi] = tdi;
          tdi += dft_tiles(D->r[2] * S.kxh, D->yiC.shape);
          ++ndi;
        }
        continue;
      }
      if (do_H) {
        YInvJob& J = Li.job[ni];
        J = YInvJob{};
        J.in = S.Z3H; J.natural = natural; J.planes = P3; J.kxh = S.kxh; J.group = group; J.fy = fy;
        J.is_C = 0; J.ny = S.ny; J.outH = S.YH;
        Li.tile_start[ni] = ti;
        ti += S.kxh * ((P3 + group - 1) / group);
        ++ni;
      }
      if (do_C) {
        YInvJob& J = Li.job[ni];
        J = YInvJob{};
        J.in = D->Z3C; J.natural = natural; J.planes = D->r[2]; J.kxh = S.kxh; J.group = group; J.fy = fy;
        J.is_C = 1; J.outC = D->YC;
        J.box_lo = D->box_lo[1]; J.box_len = D->box_len[1]; J.start = D->start[1]; J.r = D->r[1];
        J.fir = D->prefilter;
        J.periodic = periodic_axis(ctx, 1) ? 1 : 0;
        Li.tile_start[ni] = ti;
        ti += S.kxh * ((J.planes + group - 1) / group);
        ++ni;
      }
    }
    if (nf || ndf) {
      Lf.njobs = nf; Lf.tile_start[nf] = tf;
      Lz.njobs = nzj; Lz.tile_start[nzj] = tz;
      Lm.njobs = nm; Lm.tile_start[nm] = tm;
      Li.njobs = ni; Li.tile_start[ni] = ti;
      Ldf.njobs = ndf; Ldf.tile_start[ndf] = tdf;
      Ldi.njobs = ndi; Ldi.tile_start[ndi] = tdi;
      {
        Timer t(ctx, 7);
        if (ndf) CK(launch_ydft(Ldf, st));
        if (nf) CK(launch_yfwd3(Lf, st));
      }
      if (nzj) {
        Timer t(ctx, 8);
        CK(launch_zpass3(Lz, st));
      }
      if (nm) {
        Timer t(ctx, 8);
        CK(launch_zmix3(Lm, st));
      }
      Timer t(ctx, 9);
      if (ndi) CK(launch_ydft(Ldi, st));
      if (ni) CK(launch_yinv3(Li, st));
    }
  }
  {
    Launch<XInvJob> L{};
    int nj = 0, tiles = 0;
    for (int i = 0; i < n; ++i) {
      Magnet& S = ctx->mag[which[i]];
      FftTables fx;
      CKS(get_fft(ctx, S.Qx, &fx));
      if (what[i] & 1) {
        XInvJob& J = L.job[nj];
        J.in = S.YH;
        J.out = S.Hself;
        J.planes = 3 * S.nz; J.rows_per_plane = S.ny; J.kxh = S.kxh;
        J.fx = fx;
        J.box_lo = 0; J.box_len = S.nx; J.start = 0; J.out_len = S.nx; J.fir = 0;
        L.tile_start[nj] = tiles;
        tiles += (J.planes * J.rows_per_plane + kRowsPerCta - 1) / kRowsPerCta;
        ++nj;
      }
      if (what[i] & 2) {
        Dir* D = dirs[i];
        XInvJob& J = L.job[nj];
        J.in = D->YC;
        J.out = D->C;
        J.planes = D->r[2]; J.rows_per_plane = D->r[1]; J.kxh = S.kxh;
        J.fx = fx;
        J.box_lo = D->box_lo[0]; J.box_len = D->box_len[0]; J.start = D->start[0];
        J.out_len = D->r[0]; J.fir = D->prefilter;
        J.periodic = periodic_axis(ctx, 0) ? 1 : 0;
        L.tile_start[nj] = tiles;
        tiles += (J.planes * J.rows_per_plane + kRowsPerCta - 1) / kRowsPerCta;
        ++nj;
      }
      Qmax = std::max(Qmax, S.Qx);
    }
    L.njobs = nj;
    L.tile_start[nj] = tiles;
    Timer t(ctx, 2);
    CK(launch_xinv(L, Qmax, st));
  }
  return MM_OK;
}

GatherJob gather_job(mm_ctx* ctx, int s, const float* m_t, float* H) {
  const Magnet& S = ctx->mag[s];
  const Magnet& T = ctx->mag[1 - s];
  const Dir& D = S.dir;
  GatherJob J{};
  J.C = D.C;
  J.rx = D.r[0]; J.ry = D.r[1]; J.rz = D.r[2];
  J.nx = T.nx; J.ny = T.ny; J.nz = T.nz;
  J.ucell = ctx->mech->ucell[s];
  J.ufrac = ctx->mech->ufrac[s];
  for (int a = 0; a < 3; ++a) {
    J.U0[a] = D.U0[a];
    J.guard[a] = D.guard[a];
    J.inv_d[a] = (float)(1.0 / T.d[a]);
  }
  J.m = m_t;
  J.H = H;
  J.partial = D.partial;
  J.err = ctx->err_flag;
  for (int a = 0; a < 2; ++a)
    if (periodic_axis(ctx, a)) {
      const int P = a == 0 ? S.nx : S.ny;
      J.wrapP[a] = P;
      // first tap of target cell 0: source node (T.off - S.off) + floor(sigma u) - 1
      J.tap0[a] = (int)(((T.off[a] - S.off[a] - 1) % P + P) % P);
    }
  return J;
}

// P: reduction / slider update done by the gather's last block (null: none)
mm_status run_gathers(mm_ctx* ctx, const float* in[2], const int* srcs, int n, float* const* Hout) {
  CKS(join_mech(ctx));  // the gathers read the displacement
  Launch<GatherJob> L{};
  L.njobs = n;
  int tiles = 0, nzmax = 1;
  for (int i = 0; i < n; ++i) {
    const int s = srcs[i];
    L.job[i] = gather_job(ctx, s, in[1 - s], Hout[i]);
    L.tile_start[i] = tiles;
    tiles += ctx->mag[s].dir.ntiles;
    nzmax = std::max(nzmax, ctx->mag[1 - s].nz);
  }
  L.tile_start[n] = tiles;
  Timer t(ctx, 3);
  CK(launch_gather(L, nzmax, ctx->st));
  return MM_OK;
}

MechParams mech_params(mm_ctx* ctx, int mode, int stage, double dt, bool dir0, bool dir1) {
  MechParams P{};
  P.state = ctx->mech;
  const bool use[2] = {dir0, dir1};
  for (int s = 0; s < 2; ++s) {
    const Magnet& T = ctx->mag[1 - s];
    // direction s -> t: partial index s (0: base -> slider, 1: slider -> base)
    if (use[s]) {
      P.partial[s] = ctx->mag[s].dir.partial;
      P.nparts[s] = ctx->mag[s].dir.ntiles;
    }
    const double V = T.d[0] * T.d[1] * T.d[2];
    P.Fscale[s] = -kMu0 * V * T.Ms;
    P.Escale[s] = kMu0 * V * T.Ms;
    if (mode == 5) {  // only the error-norm reduction reads the stage partials
      P.err_partial[s] = ctx->mag[s].err_partial;
      P.nerr[s] = ctx->mag[s].nerr;
    }
  }
  P.mode = mode;
  P.stage = stage;
  P.dt = dt;
  if (stage >= 1 && stage < 7)
    for (int j = 0; j < 7; ++j) P.a[j] = DP_A[stage][j];
  if (mode == 2)
    for (int j = 0; j < 7; ++j) P.a[j] = DP_A[1][j];
  P.c_next = (mode == 2) ? DP_C[1] : (stage >= 1 && stage < 7 ? DP_C[stage] : 0.0);
  if (ctx->opt.integrator == MM_EULER && mode == 0 && stage == 1) {  // x + dt v, v + dt a at t + dt
    for (int j = 0; j < 7; ++j) P.a[j] = j == 0 ? 1.0 : 0.0;
    P.c_next = 1.0;
  }
  P.move = ctx->move ? 1 : 0;
  P.mass = ctx->mass;
  P.inv_mass = ctx->mass > 0 ? 1.0 / ctx->mass : 0.0;
  P.k_spring = ctx->k_spring;
  P.v_drive = ctx->v_drive;
  P.x0_spring = ctx->x0_spring;
  P.gamma_v = ctx->gamma_v;
  for (int a = 0; a < 3; ++a) {
    P.e[a] = ctx->e[a];
    P.inv_d[a] = 1.0 / ctx->mag[0].d[a];
    P.u_base[a] = ctx->u_base[a] / ctx->mag[0].d[a];
  }
  return P;
}

mm_status run_mech(mm_ctx* ctx, const MechParams& P) {
  CKS(join_mech(ctx));
  Timer t(ctx, 5);
  CK(launch_mech(P, ctx->st));
  return MM_OK;
}

// The same update on the side stream, after the work queued so far on the
// context stream, which goes on without waiting for it (join_mech waits).
mm_status fork_mech(mm_ctx* ctx, const MechParams& P) {
  CKS(join_mech(ctx));
  CK(cudaEventRecord(ctx->ev_fork, ctx->st));
  CK(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
  CK(launch_mech(P, ctx->side));
  CK(cudaEventRecord(ctx->ev_join, ctx->side));
  ctx->mech_pending = true;
  ctx->launches++;
  return MM_OK;
}

// All fields of both magnets for stage inputs `in` (demag, stray, force
// partials), then the force reduction P: for a step stage (mode 0) on the side
// stream beside the LLG stage launch, otherwise in line.
mm_status evaluate_fields(mm_ctx* ctx, const float* in[2], const MechParams& P) {
  const int which[2] = {0, 1};
  const int what[2] = {3, 3};
  Dir* dirs[2] = {&ctx->mag[0].dir, &ctx->mag[1].dir};
  CKS(run_source_passes(ctx, in, which, 2, what, dirs));
  const int srcs[2] = {0, 1};
  // H_stray of the slider comes from source 0, of the base from source 1
  float* H[2] = {ctx->mag[1].Hstray, ctx->mag[0].Hstray};
  CKS(run_gathers(ctx, in, srcs, 2, H));
  if (P.mode == 0) CKS(fork_mech(ctx, P));
  else CKS(run_mech(ctx, P));
  return MM_OK;
}

StageJob stage_job(mm_ctx* ctx, int g, const float* ys, float* ys_next, int stage, int mode, double dt,
                   float* const* kptr, float* Heff) {
  const Magnet& M = ctx->mag[g];
  StageJob J{};
  J.ys = ys;
  J.y = M.m;
  J.ys_next = ys_next;
  for (int i = 0; i < 7; ++i) J.k[i] = kptr[i];
  J.Hself = M.Hself;
  J.Hstray = M.Hstray;
  J.Heddy = M.Heddy_valid ? M.Heddy : nullptr;
  J.Heff = Heff;
  J.nx = M.nx; J.ny = M.ny; J.nz = M.nz;
  J.wrap[0] = periodic_axis(ctx, 0) ? 1 : 0;
  J.wrap[1] = periodic_axis(ctx, 1) ? 1 : 0;
  for (int a = 0; a < 3; ++a) {
    J.ex[a] = (float)(2.0 * M.Aex / (kMu0 * M.Ms * M.d[a] * M.d[a]));
    J.hext[a] = (float)ctx->Hext[a];
  }
  const double kn = sqrt(M.ku[0] * M.ku[0] + M.ku[1] * M.ku[1] + M.ku[2] * M.ku[2]);
  for (int a = 0; a < 3; ++a) J.ku[a] = (float)(kn > 0 ? M.ku[a] / kn : 0.0);
  J.an = (float)(2.0 * M.Ku / (kMu0 * M.Ms));
  J.pref = (float)(-kMu0 * kGammaLL / (1.0 + M.alpha * M.alpha));
  J.alpha = (float)M.alpha;
  J.stage = stage;
  J.mode = mode;
  if (mode == 0 && stage < 7)
    for (int j = 0; j < stage; ++j) J.comb[j] = (float)(dt * DP_A[stage][j]);
  if (mode == 0 && stage == 1 && ctx->opt.integrator == MM_EULER) J.comb[0] = (float)dt;  // y + dt k1
  if (mode == 0 && stage == 7)
    for (int j = 0; j < 7; ++j) J.ecoef[j] = (float)(dt * (DP_B5[j] - DP_B4[j]));
  J.err_partial = M.err_partial;
  return J;
}

mm_status run_stage(mm_ctx* ctx, const float* ys[2], float* ys_next[2], int stage, double dt) {
  Launch<StageJob> L{};
  L.njobs = 2;
  int tiles = 0;
  for (int g = 0; g < 2; ++g) {
    L.job[g] = stage_job(ctx, g, ys[g], ys_next[g], stage, 0, dt, ctx->mag[g].k, nullptr);
    L.tile_start[g] = tiles;
    tiles += ctx->mag[g].nerr;
  }
  L.tile_start[2] = tiles;
  // the last stage's last block reduces the embedded error norm
  const MechParams Perr = stage == 7 ? mech_params(ctx, 5, 7, dt, false, false) : MechParams{};
  Timer t(ctx, 4);
  CK(launch_stage(L, Perr, ctx->tickets + 1, ctx->st));
  return MM_OK;
}

// the device error flag: bit 1 from the gather (a target outside the box),
// bit 2 from the tensor-core DFT (a bounded wait ran out)
static mm_status device_error(mm_ctx* ctx, int e) {
  if (e & 2) return fail(ctx, MM_ETIMEOUT, "tensor-core y DFT: a wait on the MMA completion ran out");
  return fail(ctx, MM_ERANGE, "slider displacement left the planned potential box during a step");
}

mm_status check_device_error(mm_ctx* ctx) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, ctx->err_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (e) {
    CK(cudaMemsetAsync(ctx->err_flag, 0, sizeof(int), ctx->st));
    return device_error(ctx, e);
  }
  return MM_OK;
}

// Queues one step attempt of size dt and the readback of its slider state
// and range flag; attempt_finish waits for them.
mm_status attempt_enqueue(mm_ctx* ctx, double dt) {
  Magnet* M = ctx->mag;
  if (ctx->opt.integrator == MM_EULER) {
    // one field evaluation at the accepted state, y + dt f(t, y) into ys[1]
    // (the accept renormalises it into m); the slider by the same stage
    CKS(run_mech(ctx, mech_params(ctx, 4, 0, dt, false, false)));
    const float* in[2] = {M[0].m, M[1].m};
    CKS(evaluate_fields(ctx, in, mech_params(ctx, 0, 1, dt, true, true)));
    float* nxt[2] = {M[0].ys[1], M[1].ys[1]};
    CKS(run_stage(ctx, in, nxt, 1, dt));
    CKS(join_mech(ctx));
    CK(cudaMemcpyAsync(&ctx->rb->mech, ctx->mech, sizeof(MechState), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(&ctx->rb->err, ctx->err_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaEventRecord(ctx->ev_done, ctx->st));
    return MM_OK;
  }
  if (!ctx->k1_valid) {
    CKS(run_mech(ctx, mech_params(ctx, 4, 0, dt, false, false)));
    const float* in[2] = {M[0].m, M[1].m};
    CKS(evaluate_fields(ctx, in, mech_params(ctx, 0, 1, dt, true, true)));
    float* nxt[2] = {M[0].ys[0], M[1].ys[0]};
    CKS(run_stage(ctx, in, nxt, 1, dt));
  } else {
    Launch<CombineJob> L{};
    L.njobs = 2;
    int tiles = 0;
    for (int g = 0; g < 2; ++g) {
      CombineJob& J = L.job[g];
      J.y = M[g].m;
      J.out = M[g].ys[0];
      J.k[0] = M[g].k[0];
      J.comb[0] = (float)(dt * DP_A[1][0]);
      J.nk = 1;
      J.n = M[g].N;
      L.tile_start[g] = tiles;
      tiles += (int)((3 * M[g].N + 255) / 256);
    }
    L.tile_start[2] = tiles;
    {
      Timer t(ctx, 6);
      CK(launch_combine(L, ctx->st));
    }
    // the slider's stage-2 input is first read by the gathers: beside the FFT passes
    CKS(fork_mech(ctx, mech_params(ctx, 2, 1, dt, false, false)));
  }
  int cur = 0;
  for (int i = 2; i <= 7; ++i) {
    const float* in[2] = {M[0].ys[cur], M[1].ys[cur]};
    // the side stream reduces the forces and advances the slider stage
    CKS(evaluate_fields(ctx, in, mech_params(ctx, 0, i, dt, true, true)));
    float* nxt[2] = {M[0].ys[1 - cur], M[1].ys[1 - cur]};
    CKS(run_stage(ctx, in, nxt, i, dt));
    if (i < 7) cur = 1 - cur;
  }
  // stages 2..7 alternate the two stage buffers, so the stage-7 input (the
  // 5th-order solution) always ends in ys[1]
  (void)cur;
  CKS(join_mech(ctx));
  CK(cudaMemcpyAsync(&ctx->rb->mech, ctx->mech, sizeof(MechState), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(&ctx->rb->err, ctx->err_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaEventRecord(ctx->ev_done, ctx->st));
  return MM_OK;
}

// Waits for the attempt queued by attempt_enqueue; its error norm in *err.
mm_status attempt_finish(mm_ctx* ctx, double* err) {
  CK(cudaEventSynchronize(ctx->ev_done));
  ctx->host_mech = ctx->rb->mech;
  if (ctx->rb->err) {
    const int e = ctx->rb->err;
    ctx->rb->err = 0;
    CK(cudaMemsetAsync(ctx->err_flag, 0, sizeof(int), ctx->st));
    return device_error(ctx, e);
  }
  *err = ctx->host_mech.err;
  return MM_OK;
}

// Step-size control after an attempt with error norm err: on acceptance the
// new m, the slider state and the first-same-as-last k1 are committed (and
// the plan follows a whole-cell move); dt becomes the next attempt's size.
mm_status conclude_attempt(mm_ctx* ctx, double* dt_io, double err, bool* accepted) {
  double dt = *dt_io;
  const bool accept = !ctx->opt.adaptive || err <= ctx->opt.rtol || dt <= ctx->opt.dt_min;
  if (ctx->attempts.size() >= (size_t)kAttemptLog) ctx->attempts.pop_front();
  ctx->attempts.push_back({ctx->host_mech.t, dt, err, accept ? 1 : 0});
  double fac = 5.0;
  if (err > 0.0) fac = std::min(5.0, std::max(0.2, 0.9 * pow(ctx->opt.rtol / err, 0.2)));
  if (accept) {
    Launch<CombineJob> L{};
    L.njobs = 2;
    int tiles = 0;
    for (int g = 0; g < 2; ++g) {
      CombineJob& J = L.job[g];
      // after an attempt the 5th-order solution is in ys[1] (stages 2..7 alternate 0,1,0,1,0,1)
      J.y = ctx->mag[g].ys[1];
      J.out = ctx->mag[g].m;
      J.n = ctx->mag[g].N;
      L.tile_start[g] = tiles;
      tiles += (int)((ctx->mag[g].N + 255) / 256);
    }
    L.tile_start[2] = tiles;
    {
      Timer t(ctx, 6);
      CK(launch_normalise(L, ctx->st));
    }
    // conducting magnets: B of this step's last evaluation (the stage-7 fields
    // at the 5th-order solution ys[1]), its rate since the last step, and the
    // eddy field the next step's stages add to H_eff (lagged by one step)
    // (the currents of a conducting magnet also act on the other magnet: their
    // field there is added to that magnet's eddy field below, whether or not
    // it conducts)
    bool own[2] = {false, false};
    for (int g = 0; g < 2; ++g) {
      Magnet& M = ctx->mag[g];
      if (!(M.sigma > 0.0)) continue;
      CKS(ensure_buf(ctx, &M.Bprev, &M.eb_bytes[0], sizeof(float) * 3 * M.N));
      CKS(ensure_buf(ctx, &M.Bdot, &M.eb_bytes[1], sizeof(float) * 3 * M.N));
      CKS(ensure_buf(ctx, &M.Heddy, &M.eb_bytes[2], sizeof(float) * 3 * M.N));
      CK(launch_flux_rate(M.Hself, M.Hstray, M.ys[1], M.N, ctx->Hext, M.Ms, dt, M.B_valid ? 1 : 0, M.Bprev, M.Bdot,
                          ctx->st));
      if (M.B_valid) {
        CKS(eddy_core(ctx, g, M.Bdot, M.sigma, M.Heddy, nullptr, nullptr));  // J in M.ed_J
        own[g] = true;
        M.Heddy_valid = true;
      }
      M.B_valid = true;
    }
    const bool fsal = ctx->opt.integrator == MM_RK45;  // Euler evaluates afresh every step
    if (fsal)
      for (int g = 0; g < 2; ++g) std::swap(ctx->mag[g].k[0], ctx->mag[g].k[6]);
    // the accepted slider state, beside the normalisation
    CKS(fork_mech(ctx, mech_params(ctx, 3, 7, dt, false, false)));
    ctx->host_mech.x = ctx->host_mech.xs;
    ctx->host_mech.v = ctx->host_mech.vs;
    ctx->host_mech.t = ctx->host_mech.t + dt;
    ctx->host_mech.kx[0] = ctx->host_mech.kx[6];
    ctx->host_mech.kv[0] = ctx->host_mech.kv[6];
    ctx->k1_valid = fsal;
    ctx->accepted++;
    // the field of each conducting magnet's currents inside the other, at the
    // accepted displacement (that of the step's last evaluation)
    for (int t = 0; t < 2; ++t) {
      const int g = 1 - t;
      if (!own[g]) continue;
      Magnet& T = ctx->mag[t];
      CKS(ensure_buf(ctx, &T.Heddy, &T.eb_bytes[2], sizeof(float) * 3 * T.N));
      if (own[t]) {
        CKS(ensure_buf(ctx, &T.ex_H, &T.ex_bytes[1], sizeof(float) * 3 * T.N));
        CKS(cross_eddy_field(ctx, g, ctx->mag[g].ed_J, T.ex_H));
        CK(launch_accumulate(T.ex_H, 3 * T.N, T.Heddy, ctx->st));
      } else {
        CKS(cross_eddy_field(ctx, g, ctx->mag[g].ed_J, T.Heddy));
      }
      T.Heddy_valid = true;
    }
    // a whole-cell move beyond the guard needs new boxes (and a fresh k1)
    bool moved = false;
    for (int s = 0; s < 2 && !moved; ++s)
      for (int a = 0; a < 3; ++a) {
        if (periodic_axis(ctx, a)) continue;
        const double sigma = s == 0 ? 1.0 : -1.0;
        if ((int)floor(sigma * u_cells(ctx, a, ctx->host_mech.x)) != ctx->mag[s].dir.U0[a]) moved = true;
      }
    if (moved) {
      CKS(ensure_plan(ctx));
      CKS(upload_mech(ctx));
      ctx->k1_valid = false;
    }
  } else {
    ctx->rejected++;
  }
  if (ctx->opt.adaptive) dt = std::min(std::max(dt * fac, ctx->opt.dt_min), ctx->opt.dt_max);
  *dt_io = dt;
  *accepted = accept;
  return MM_OK;
}

}  // namespace

// ============================================================ C ABI
extern "C" {

void mm_default_options(mm_options* o) {
  if (!o) return;
  o->precision = MM_FP32;
  o->margin = 4;
  o->adaptive = 1;
  o->rtol = 1e-5;
  o->dt_min = 1e-16;
  o->dt_max = 1e-11;
  o->stream = nullptr;
  o->periodic = 0;
  o->pbc_images = 2;
  o->integrator = MM_RK45;
}

const char* mm_status_string(mm_status s) {
  switch (s) {
    case MM_OK: return "ok";
    case MM_EINVAL: return "invalid argument";
    case MM_ENOMEM: return "out of device memory";
    case MM_ECUDA: return "CUDA error";
    case MM_ERANGE: return "displacement outside planned box";
    case MM_ETIMEOUT: return "timeout";
    case MM_ESTATE: return "bad state buffer";
    case MM_ENOTSUP: return "not supported";
    case MM_ETOOBIG: return "larger than the fixed scratch of the no-allocation entry point";
  }
  return "unknown";
}

mm_status mm_create(mm_ctx** out, const mm_options* opt) {
  if (!out) return MM_EINVAL;
  *out = nullptr;
  mm_ctx* ctx = new mm_ctx();
  if (opt) ctx->opt = *opt;
  else mm_default_options(&ctx->opt);
  if (ctx->opt.precision != MM_FP32 && ctx->opt.precision != MM_MIXED) {
    delete ctx;
    return MM_ENOTSUP;
  }
  if (ctx->opt.margin < 0 || ctx->opt.margin > 64 || ctx->opt.periodic < 0 || ctx->opt.periodic > 3 ||
      ctx->opt.pbc_images < 0 || ctx->opt.pbc_images > 64 ||
      (ctx->opt.integrator != MM_RK45 && ctx->opt.integrator != MM_EULER) ||
      (ctx->opt.integrator == MM_EULER && ctx->opt.adaptive)) {
    delete ctx;
    return MM_EINVAL;
  }
  ctx->st = (cudaStream_t)ctx->opt.stream;
  cudaError_t e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->rb, sizeof(mm_ctx::Readback));
  if (e == cudaSuccess) memset(ctx->rb, 0, sizeof(mm_ctx::Readback));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->mech, sizeof(MechState));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->err_flag, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->tickets, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->tickets, 0, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->err_flag, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->mech, 0, sizeof(MechState));
  if (e == cudaSuccess) e = init_fft_constants_passes();
  if (e == cudaSuccess) e = init_fft_constants_kgen();
  if (e == cudaSuccess) e = init_fft_constants_3d();
  if (e != cudaSuccess) {
    mm_destroy(ctx);
    return e == cudaErrorMemoryAllocation ? MM_ENOMEM : MM_ECUDA;
  }
  *out = ctx;
  return MM_OK;
}

static void free_dft(DftMat& M) {
  cudaFree(M.hi); cudaFree(M.lo);
  M = DftMat();
}

static void free_dir(Dir& D) {
  cudaFree(D.Tq); cudaFree(D.YC); cudaFree(D.C); cudaFree(D.partial); cudaFree(D.Z3C); cudaFree(D.pkC);
  free_dft(D.yiC);
  D = Dir();
}

void mm_destroy(mm_ctx* ctx) {
  if (!ctx) return;
  if (ctx->side) cudaStreamSynchronize(ctx->side);
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  else cudaDeviceSynchronize();
  for (auto& M : ctx->mag) {
    cudaFree(M.m);
    for (auto p : M.ys) cudaFree(p);
    for (auto p : M.k) cudaFree(p);
    cudaFree(M.Hself); cudaFree(M.Hstray); cudaFree(M.scratch3); cudaFree(M.err_partial);
    cudaFree(M.pow_H); cudaFree(M.pow_part);
    cudaFree(M.X1); cudaFree(M.YH); cudaFree(M.Nq);
    cudaFree(M.N3); cudaFree(M.S3); cudaFree(M.Y3); cudaFree(M.Z3H);
    free_dft(M.yf); free_dft(M.yiH); cudaFree(M.pkH); cudaFree(M.pkX);
    cudaFree(M.adj_box); cudaFree(M.adj_grid); cudaFree(M.adj_X); cudaFree(M.adj_Y); cudaFree(M.adj_Z);
    cudaFree(M.adj_YH); cudaFree(M.adj_Sq);
    free_dir(M.dir);
    free_dir(M.aux);
    free_dir(M.cw);
    cudaFree(M.cw_Y);
    free_dir(M.eddy);
    free_dir(M.eddyx);
    cudaFree(M.ex_C3); cudaFree(M.ex_H);
    cudaFree(M.ed_V); cudaFree(M.ed_E); cudaFree(M.ed_b); cudaFree(M.ed_phi); cudaFree(M.ed_J);
    cudaFree(M.ed_part); cudaFree(M.ed_stats);
    cudaFree(M.Bprev); cudaFree(M.Bdot); cudaFree(M.Heddy);
  }
  for (auto& kv : ctx->ffts) {
    cudaFree(kv.second.tw_f); cudaFree(kv.second.tw_d); cudaFree(kv.second.pos); cudaFree(kv.second.freq);
  }
  cudaFree(ctx->gen_work); cudaFree(ctx->gen_q); cudaFree(ctx->W_dev); cudaFree(ctx->dc_buf);
  cudaFree(ctx->fd4_C); cudaFree(ctx->fd4_V);
  cudaFree(ctx->mech); cudaFree(ctx->err_flag); cudaFree(ctx->tickets);
  for (auto& p : ctx->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->ev_done) cudaEventDestroy(ctx->ev_done);
  if (ctx->rb) cudaFreeHost(ctx->rb);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  for (auto e : ctx->free_events) cudaEventDestroy(e);
  delete ctx;
}

const char* mm_last_error(const mm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

static bool bad_mag(int mag) { return mag != 0 && mag != 1; }

mm_status mm_set_grid(mm_ctx* ctx, int mag, int nx, int ny, int nz, double dx, double dy, double dz,
                      const long long offset_cells[3]) {
  if (!ctx) return MM_EINVAL;
  if (bad_mag(mag) || nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dy > 0) || !(dz > 0) || !offset_cells)
    return fail(ctx, MM_EINVAL, "mm_set_grid: bad argument");
  if ((long long)nx * ny * nz > (1ll << 30)) return fail(ctx, MM_ENOTSUP, "mm_set_grid: more than 2^30 cells");
  const Magnet& O = ctx->mag[1 - mag];
  if (O.grid && (O.d[0] != dx || O.d[1] != dy || O.d[2] != dz))
    return fail(ctx, MM_EINVAL, "mm_set_grid: both magnets must share the cell size");
  Magnet& M = ctx->mag[mag];
  if (M.grid && (M.nx != nx || M.ny != ny || M.nz != nz))
    return fail(ctx, MM_EINVAL, "mm_set_grid: grid size is fixed once set");
  M.nx = nx; M.ny = ny; M.nz = nz;
  M.N = (size_t)nx * ny * nz;
  M.d[0] = dx; M.d[1] = dy; M.d[2] = dz;
  for (int a = 0; a < 3; ++a) M.off[a] = offset_cells[a];
  M.grid = true;
  CKS(alloc_magnet(ctx, M));
  ctx->planned = false;
  ctx->k1_valid = false;
  return MM_OK;
}

mm_status mm_set_material(mm_ctx* ctx, int mag, double Ms, double Aex, double Ku, const double ku_axis[3],
                          double alpha) {
  if (ctx) reset_eddy(ctx);
  if (!ctx) return MM_EINVAL;
  if (bad_mag(mag) || !(Ms > 0) || Aex < 0 || alpha < 0 || !ku_axis)
    return fail(ctx, MM_EINVAL, "mm_set_material: bad argument");
  Magnet& M = ctx->mag[mag];
  M.Ms = Ms; M.Aex = Aex; M.Ku = Ku; M.alpha = alpha;
  for (int a = 0; a < 3; ++a) M.ku[a] = ku_axis[a];
  M.mat = true;
  ctx->planned = false;
  ctx->k1_valid = false;
  // spectra carry Ms: force a rebuild of this source's kernels
  M.Nq_Ms = 0;
  M.dir.Tq_prefilter = -1;
  M.aux.Tq_prefilter = -1;
  return MM_OK;
}

mm_status mm_set_external_field(mm_ctx* ctx, const double H[3]) {
  if (ctx) reset_eddy(ctx);
  if (!ctx || !H) return MM_EINVAL;
  for (int a = 0; a < 3; ++a) ctx->Hext[a] = H[a];
  ctx->k1_valid = false;
  return MM_OK;
}

mm_status mm_set_mechanics(mm_ctx* ctx, double mass, double k_spring, double v_drive, double gamma_visc,
                           const double drive_dir[3], double x0_spring) {
  if (!ctx || !drive_dir) return MM_EINVAL;
  const double n = sqrt(drive_dir[0] * drive_dir[0] + drive_dir[1] * drive_dir[1] + drive_dir[2] * drive_dir[2]);
  if (!(n > 0)) return fail(ctx, MM_EINVAL, "mm_set_mechanics: zero drive direction");
  ctx->move = mass > 0;
  ctx->mass = mass; ctx->k_spring = k_spring; ctx->v_drive = v_drive; ctx->gamma_v = gamma_visc;
  ctx->x0_spring = x0_spring;
  for (int a = 0; a < 3; ++a) ctx->e[a] = drive_dir[a] / n;
  ctx->planned = false;
  ctx->k1_valid = false;
  return MM_OK;
}

mm_status mm_set_magnetization(mm_ctx* ctx, int mag, const float* m_dev) {
  if (ctx) reset_eddy(ctx);
  if (!ctx || bad_mag(mag) || !m_dev) return ctx ? fail(ctx, MM_EINVAL, "mm_set_magnetization") : MM_EINVAL;
  Magnet& M = ctx->mag[mag];
  if (!M.grid) return fail(ctx, MM_EINVAL, "mm_set_magnetization: grid not set");
  CK(cudaMemcpyAsync(M.m, m_dev, sizeof(float) * 3 * M.N, cudaMemcpyDeviceToDevice, ctx->st));
  M.mset = true;
  ctx->k1_valid = false;
  return MM_OK;
}

mm_status mm_get_magnetization(mm_ctx* ctx, int mag, float* m_dev) {
  if (!ctx || bad_mag(mag) || !m_dev) return ctx ? fail(ctx, MM_EINVAL, "mm_get_magnetization") : MM_EINVAL;
  Magnet& M = ctx->mag[mag];
  if (!M.grid) return fail(ctx, MM_EINVAL, "mm_get_magnetization: grid not set");
  CK(cudaMemcpyAsync(m_dev, M.m, sizeof(float) * 3 * M.N, cudaMemcpyDeviceToDevice, ctx->st));
  return MM_OK;
}

mm_status mm_upload_magnetization(mm_ctx* ctx, int mag, const float* m_host) {
  if (ctx) reset_eddy(ctx);
  if (!ctx || bad_mag(mag) || !m_host) return ctx ? fail(ctx, MM_EINVAL, "mm_upload_magnetization") : MM_EINVAL;
  Magnet& M = ctx->mag[mag];
  if (!M.grid) return fail(ctx, MM_EINVAL, "mm_upload_magnetization: grid not set");
  CK(cudaMemcpyAsync(M.m, m_host, sizeof(float) * 3 * M.N, cudaMemcpyHostToDevice, ctx->st));
  M.mset = true;
  ctx->k1_valid = false;
  return MM_OK;
}

mm_status mm_download_magnetization(mm_ctx* ctx, int mag, float* m_host) {
  if (!ctx || bad_mag(mag) || !m_host) return ctx ? fail(ctx, MM_EINVAL, "mm_download_magnetization") : MM_EINVAL;
  Magnet& M = ctx->mag[mag];
  if (!M.grid) return fail(ctx, MM_EINVAL, "mm_download_magnetization: grid not set");
  CK(cudaMemcpyAsync(m_host, M.m, sizeof(float) * 3 * M.N, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return MM_OK;
}

mm_status mm_set_displacement(mm_ctx* ctx, const double u_m[3]) {
  if (ctx) reset_eddy(ctx);
  if (!ctx || !u_m) return MM_EINVAL;
  for (int a = 0; a < 3; ++a) {
    if (!isfinite(u_m[a])) return fail(ctx, MM_EINVAL, "mm_set_displacement: non-finite");
    ctx->u_base[a] = u_m[a];
  }
  ctx->host_mech.x = 0.0;
  ctx->k1_valid = false;
  if (ctx->planned) CKS(replan_if_needed(ctx));
  return MM_OK;
}

mm_status mm_set_slider_state(mm_ctx* ctx, double x, double v, double t) {
  if (ctx) reset_eddy(ctx);
  if (!ctx) return MM_EINVAL;
  ctx->host_mech.x = x; ctx->host_mech.v = v; ctx->host_mech.t = t;
  ctx->k1_valid = false;
  if (ctx->planned) CKS(replan_if_needed(ctx));
  return MM_OK;
}

mm_status mm_get_slider_state(mm_ctx* ctx, double* x, double* v, double* t) {
  if (!ctx) return MM_EINVAL;
  if (x) *x = ctx->host_mech.x;
  if (v) *v = ctx->host_mech.v;
  if (t) *t = ctx->host_mech.t;
  return MM_OK;
}

static mm_status prepare(mm_ctx* ctx) {
  if (!ctx->mag[0].mset || !ctx->mag[1].mset) return fail(ctx, MM_EINVAL, "magnetisation not set");
  CKS(replan_if_needed(ctx));
  // while a first-same-as-last k1 is held the device slider state is the
  // authoritative one; any set_* call clears k1_valid and re-uploads
  if (!ctx->k1_valid) CKS(upload_mech(ctx));
  return MM_OK;
}

mm_status mm_compute_fields(mm_ctx* ctx) {
  if (!ctx) return MM_EINVAL;
  CKS(prepare(ctx));
  const float* in[2] = {ctx->mag[0].m, ctx->mag[1].m};
  CKS(evaluate_fields(ctx, in, mech_params(ctx, 1, 0, 0.0, true, true)));
  return MM_OK;
}

mm_status mm_compute_stray_field(mm_ctx* ctx, int src, float* H_dev) {
  if (!ctx || bad_mag(src)) return ctx ? fail(ctx, MM_EINVAL, "mm_compute_stray_field") : MM_EINVAL;
  CKS(prepare(ctx));
  const float* in[2] = {ctx->mag[0].m, ctx->mag[1].m};
  const int which[1] = {src};
  const int what[1] = {2};
  Dir* dirs[1] = {&ctx->mag[src].dir};
  CKS(run_source_passes(ctx, in, which, 1, what, dirs));
  float* H[1] = {H_dev ? H_dev : ctx->mag[1 - src].Hstray};
  const MechParams P = mech_params(ctx, 1, 0, 0.0, src == 0, src == 1);
  CKS(run_gathers(ctx, in, which, 1, H));
  CKS(run_mech(ctx, P));
  return MM_OK;
}

mm_status mm_backward_energy(mm_ctx* ctx, int src, double dE_du[3], float* dE_dm_src_dev,
                             float* dE_dm_tgt_dev) {
  if (ctx && ctx->opt.periodic) return fail(ctx, MM_ENOTSUP, "mm_backward_energy: periodic boundaries");
  if (!ctx || bad_mag(src)) return ctx ? fail(ctx, MM_EINVAL, "mm_backward_energy") : MM_EINVAL;
  // forward: potential box, stray field at the target, force and energy
  CKS(mm_compute_stray_field(ctx, src, nullptr));
  const int t = 1 - src;
  Magnet& S = ctx->mag[src];
  const Magnet& T = ctx->mag[t];
  const Dir& D = S.dir;
  cudaStream_t st = ctx->st;
  const double escale = kMu0 * T.d[0] * T.d[1] * T.d[2] * T.Ms;
  // dE/dm_t = mu0 V Ms_t grad phi = -mu0 V Ms_t H
  if (dE_dm_tgt_dev) CK(launch_scale(T.Hstray, dE_dm_tgt_dev, 3 * T.N, (float)(-escale), st));
  if (dE_dm_src_dev) {
    const int* bd = D.box_len;
    const int bz = bd[2];
    const int nzg = 3 * ((bz + 2) / 3);  // grid planes for the x pass (whole groups of three)
    const int P3 = 3 * S.nz;
    const size_t nbox = (size_t)bd[0] * bd[1] * bd[2];
    CKS(ensure_buf(ctx, &S.adj_box, &S.adj_bytes[0], sizeof(float) * nbox));
    CKS(ensure_buf(ctx, &S.adj_grid, &S.adj_bytes[1], sizeof(float) * (size_t)nzg * S.Qy * S.Qx));
    CKS(ensure_buf(ctx, &S.adj_X, &S.adj_bytes[2], sizeof(float2) * (size_t)nzg * S.kxh * S.Qy));
    CKS(ensure_buf(ctx, &S.adj_Y, &S.adj_bytes[3], sizeof(float2) * (size_t)bz * S.kxh * S.Qy));
    CKS(ensure_buf(ctx, &S.adj_Z, &S.adj_bytes[4], sizeof(float2) * (size_t)P3 * S.kxh * S.Qy));
    CKS(ensure_buf(ctx, &S.adj_YH, &S.adj_bytes[5], sizeof(float2) * (size_t)P3 * S.kxh * S.ny));
    // S spectra of every z offset between a source layer and a box plane
    const int dz_lo = D.box_lo[2] - (S.nz - 1), np = bz + S.nz - 1;
    const size_t qsize = (size_t)S.kxh * S.kyq;
    if (!S.adj_Sq || S.adj_key[0] != dz_lo || S.adj_key[1] != np || S.adj_key[2] != S.Qx ||
        S.adj_key[3] != S.Qy || S.adj_Ms != S.Ms) {
      CKS(ensure_buf(ctx, &S.adj_Sq, &S.adj_bytes[6], sizeof(float) * (size_t)np * 3 * qsize));
      FftTables fx, fy;
      CKS(get_fft(ctx, S.Qx, &fx));
      CKS(get_fft(ctx, S.Qy, &fy));
      CKS(ensure_buf(ctx, &ctx->gen_work, &ctx->gen_work_bytes, sizeof(double2) * 2 * 6 * (size_t)S.Qx * S.Qy));
      CKS(ensure_buf(ctx, &ctx->gen_q, &ctx->gen_q_bytes, std::max(ctx->gen_q_bytes, sizeof(double) * 6 * qsize)));
      const KernelPlan K{S.Qx, S.Qy, S.Wx, S.Wy, S.nz};
      CK(build_S_planes(K, fx, fy, S.d[0], S.d[1], S.d[2], S.Ms / ((double)S.Qx * S.Qy), dz_lo, np, S.adj_Sq,
                        ctx->gen_work, ctx->gen_q, st));
      CK(cudaStreamSynchronize(st));
      S.adj_key[0] = dz_lo; S.adj_key[1] = np; S.adj_key[2] = S.Qx; S.adj_key[3] = S.Qy;
      S.adj_Ms = S.Ms;
    }
    CKS(join_mech(ctx));  // the scatter reads the displacement
    // 1. transposed evaluation into the box
    CK(cudaMemsetAsync(S.adj_box, 0, sizeof(float) * nbox, st));
    AdjScatterJob A{};
    A.m = T.m;
    A.nx = T.nx; A.ny = T.ny; A.nz = T.nz;
    A.u = ctx->mech->u;
    A.sigma = src == 0 ? 1.0 : -1.0;
    for (int a = 0; a < 3; ++a) {
      A.U0[a] = D.U0[a];
      A.guard[a] = D.guard[a];
      A.inv_d[a] = (float)(1.0 / T.d[a]);
      A.bdim[a] = bd[a];
      A.start[a] = D.start[a];
      A.r[a] = D.r[a];
    }
    A.escale = (float)escale;
    A.box = S.adj_box;
    A.err = ctx->err_flag;
    CK(launch_adj_scatter(A, st));
    // 2. transposed prefilter
    CK(launch_pref_T(S.adj_box, bd, st));
    // 3. transposed potential sum: onto the circular grid, x and y forward,
    //    conjugate S spectra per source layer, y and x inverse
    CK(cudaMemsetAsync(S.adj_grid, 0, sizeof(float) * (size_t)nzg * S.Qy * S.Qx, st));
    CK(launch_place(S.adj_box, bd, D.box_lo, S.adj_grid, S.Qx, S.Qy, st));
    FftTables fx, fy;
    CKS(get_fft(ctx, S.Qx, &fx));
    CKS(get_fft(ctx, S.Qy, &fy));
    {
      Launch<XFwdJob> L{};
      L.njobs = 1;
      XFwdJob& X = L.job[0];
      X.m = S.adj_grid; X.out = S.adj_X; X.nx = S.Qx; X.ny = S.Qy; X.nz = nzg / 3; X.kxh = S.kxh; X.fx = fx;
      L.tile_start[1] = (nzg * S.Qy + kRowsPerCta - 1) / kRowsPerCta;
      CK(launch_xfwd(L, S.Qx, st));
    }
    const int group = std::max(1, std::min(16, (int)((48 * 1024) / ((S.Qy + 1) * sizeof(float2)))));
    {
      Launch<YFwdJob> L{};
      L.njobs = 1;
      YFwdJob& F = L.job[0];
      F.in = S.adj_X; F.out = S.adj_Y; F.planes = bz; F.ny = S.Qy; F.kxh = S.kxh; F.group = group;
      F.natural = 1; F.fy = fy;
      L.tile_start[1] = S.kxh * ((bz + group - 1) / group);
      CK(launch_yfwd3(L, st));
    }
    {
      ZAdjJob Z{};
      Z.in = S.adj_Y; Z.bz = bz; Z.nz = S.nz; Z.kxh = S.kxh; Z.Qy = S.Qy; Z.kyq = S.kyq;
      Z.Sq = S.adj_Sq; Z.out = S.adj_Z;
      CK(launch_zadj(Z, st));
    }
    {
      Launch<YInvJob> L{};
      L.njobs = 1;
      YInvJob& J = L.job[0];
      J.in = S.adj_Z; J.natural = 1; J.planes = P3; J.kxh = S.kxh; J.group = group; J.fy = fy;
      J.is_C = 0; J.ny = S.ny; J.outH = S.adj_YH;
      L.tile_start[1] = S.kxh * ((P3 + group - 1) / group);
      CK(launch_yinv3(L, st));
    }
    {
      Launch<XInvJob> L{};
      L.njobs = 1;
      XInvJob& J = L.job[0];
      J.in = S.adj_YH; J.out = dE_dm_src_dev;
      J.planes = P3; J.rows_per_plane = S.ny; J.kxh = S.kxh; J.fx = fx;
      J.box_lo = 0; J.box_len = S.nx; J.start = 0; J.out_len = S.nx; J.fir = 0;
      L.tile_start[1] = (P3 * S.ny + kRowsPerCta - 1) / kRowsPerCta;
      CK(launch_xinv(L, S.Qx, st));
    }
    ctx->launches += 11;
  }
  // dE/du = -sigma F_t (sigma = +1 when the target is the slider)
  CKS(join_mech(ctx));
  CK(cudaMemcpyAsync(&ctx->host_mech, ctx->mech, sizeof(MechState), cudaMemcpyDeviceToHost, ctx->st));
  CKS(check_device_error(ctx));
  if (dE_du) {
    const double* F = t == 1 ? ctx->host_mech.F_slider : ctx->host_mech.F_base;
    const double sigma = t == 1 ? 1.0 : -1.0;
    for (int a = 0; a < 3; ++a) dE_du[a] = -sigma * F[a];
  }
  return MM_OK;
}

mm_status mm_compute_demag(mm_ctx* ctx, int mag, float* H_dev) {
  if (!ctx || bad_mag(mag)) return ctx ? fail(ctx, MM_EINVAL, "mm_compute_demag") : MM_EINVAL;
  CKS(prepare(ctx));
  const float* in[2] = {ctx->mag[0].m, ctx->mag[1].m};
  const int which[1] = {mag};
  const int what[1] = {1};
  Dir* dirs[1] = {&ctx->mag[mag].dir};
  CKS(run_source_passes(ctx, in, which, 1, what, dirs));
  if (H_dev)
    CK(cudaMemcpyAsync(H_dev, ctx->mag[mag].Hself, sizeof(float) * 3 * ctx->mag[mag].N,
                       cudaMemcpyDeviceToDevice, ctx->st));
  return MM_OK;
}

mm_status mm_compute_potential(mm_ctx* ctx, int src, int prefiltered, float* out_dev, size_t capacity,
                               int dims[3], long long lo[3]) {
  if (!ctx || bad_mag(src)) return ctx ? fail(ctx, MM_EINVAL, "mm_compute_potential") : MM_EINVAL;
  if (!ctx->mag[0].grid || !ctx->mag[1].grid) return fail(ctx, MM_EINVAL, "grids not set");
  if (!ctx->mag[0].mat || !ctx->mag[1].mat) return fail(ctx, MM_EINVAL, "materials not set");
  CKS(replan_if_needed(ctx));
  Magnet& S = ctx->mag[src];
  Dir& D = S.aux;
  dir_geometry(ctx, src, true, &D);
  D.prefilter = prefiltered ? 1 : 0;
  if (dims)
    for (int a = 0; a < 3; ++a) dims[a] = D.box_len[a];
  if (lo)
    for (int a = 0; a < 3; ++a) lo[a] = D.box_lo[a];
  if (!out_dev) return MM_OK;
  const size_t need = (size_t)D.box_len[0] * D.box_len[1] * D.box_len[2];
  if (capacity < need) return fail(ctx, MM_EINVAL, "mm_compute_potential: output too small");
  if (!S.mset) return fail(ctx, MM_EINVAL, "magnetisation not set");
  if (!S.thick && (size_t)std::max(3 * S.nz, D.r[2]) * S.Qy * sizeof(float2) > 220 * 1024)
    return fail(ctx, MM_ENOTSUP, "box too tall for the fused y pass");
  if (!S.zfft) CKS(build_T(ctx, src, &D));
  if (S.thick) CKS(ensure_buf(ctx, &D.Z3C, &D.Z3C_bytes, sizeof(float2) * (size_t)D.r[2] * S.kxh * S.Qy));
  CKS(ensure_buf(ctx, &D.YC, &D.YC_bytes, sizeof(float2) * (size_t)D.r[2] * S.kxh * D.r[1]));
  const float* in[2] = {ctx->mag[0].m, ctx->mag[1].m};
  const int which[1] = {src};
  const int what[1] = {2};
  float* saveC = D.C;
  D.C = out_dev;  // x pass writes the box straight into the caller's buffer
  Dir* dirs[1] = {&D};
  mm_status s = run_source_passes(ctx, in, which, 1, what, dirs);
  D.C = saveC;
  D.valid = true;
  return s;
}

mm_status mm_get_force(mm_ctx* ctx, int on_mag, double F_out[3], double* E_int_out) {
  if (!ctx || bad_mag(on_mag)) return ctx ? fail(ctx, MM_EINVAL, "mm_get_force") : MM_EINVAL;
  CKS(join_mech(ctx));
  CK(cudaMemcpyAsync(&ctx->host_mech, ctx->mech, sizeof(MechState), cudaMemcpyDeviceToHost, ctx->st));
  CKS(check_device_error(ctx));
  const MechState& H = ctx->host_mech;
  for (int a = 0; a < 3; ++a)
    if (F_out) F_out[a] = on_mag == 1 ? H.F_slider[a] : H.F_base[a];
  if (E_int_out) *E_int_out = on_mag == 1 ? H.E_slider : H.E_base;
  return MM_OK;
}

mm_status mm_compute_torque(mm_ctx* ctx, int mag, float* dmdt_dev, float* Heff_dev) {
  if (!ctx || bad_mag(mag)) return ctx ? fail(ctx, MM_EINVAL, "mm_compute_torque") : MM_EINVAL;
  CKS(mm_compute_fields(ctx));
  Magnet& M = ctx->mag[mag];
  float* kp[7];
  for (int i = 0; i < 7; ++i) kp[i] = M.k[i];
  kp[0] = dmdt_dev ? dmdt_dev : M.scratch3;
  Launch<StageJob> L{};
  L.njobs = 1;
  L.job[0] = stage_job(ctx, mag, M.m, nullptr, 1, 1, 0.0, kp, Heff_dev);
  L.tile_start[0] = 0;
  L.tile_start[1] = M.nerr;
  {
    Timer t(ctx, 4);
    CK(launch_stage(L, MechParams{}, nullptr, ctx->st));
  }
  ctx->k1_valid = false;
  return MM_OK;
}

mm_status mm_get_power(mm_ctx* ctx, double* P_in, double P_diss[2], double* P_visc) {
  if (!ctx) return MM_EINVAL;
  CKS(mm_compute_fields(ctx));
  for (int g = 0; g < 2; ++g) {
    Magnet& M = ctx->mag[g];
    CKS(ensure_buf(ctx, &M.pow_H, &M.pow_H_bytes, sizeof(float) * 3 * M.N));
    CKS(ensure_buf(ctx, &M.pow_part, &M.pow_part_bytes, sizeof(double) * (power_blocks(M.N) + 1)));
    float* kp[7];
    for (int i = 0; i < 7; ++i) kp[i] = M.k[i];
    kp[0] = M.scratch3;  // the torque itself is not kept
    Launch<StageJob> L{};
    L.njobs = 1;
    L.job[0] = stage_job(ctx, g, M.m, nullptr, 1, 1, 0.0, kp, M.pow_H);
    L.tile_start[0] = 0;
    L.tile_start[1] = M.nerr;
    {
      Timer t(ctx, 4);
      CK(launch_stage(L, MechParams{}, nullptr, ctx->st));
    }
    // the sum lands after the block sums
    CK(launch_mxh2(M.m, M.pow_H, M.N, M.pow_part, M.pow_part + power_blocks(M.N), ctx->st));
  }
  ctx->k1_valid = false;
  double S[2] = {0.0, 0.0};
  for (int g = 0; g < 2; ++g)
    CK(cudaMemcpyAsync(&S[g], ctx->mag[g].pow_part + power_blocks(ctx->mag[g].N), sizeof(double),
                       cudaMemcpyDeviceToHost, ctx->st));
  CKS(join_mech(ctx));
  CK(cudaMemcpyAsync(&ctx->host_mech, ctx->mech, sizeof(MechState), cudaMemcpyDeviceToHost, ctx->st));
  CKS(check_device_error(ctx));
  const MechState& H = ctx->host_mech;
  const double v = ctx->move ? H.v : 0.0;
  const double Fe = H.F_slider[0] * ctx->e[0] + H.F_slider[1] * ctx->e[1] + H.F_slider[2] * ctx->e[2];
  if (P_in) *P_in = -Fe * v;
  for (int g = 0; g < 2; ++g) {
    const Magnet& M = ctx->mag[g];
    const double V = M.d[0] * M.d[1] * M.d[2];
    const double a = M.alpha;
    if (P_diss) P_diss[g] = kMu0 * kGammaLL * a * kMu0 * V * M.Ms / (1.0 + a * a) * S[g];
  }
  if (P_visc) *P_visc = ctx->move ? ctx->gamma_v * ctx->mass * v * v : 0.0;
  return MM_OK;
}

mm_status mm_compute_stray_field_fd4(mm_ctx* ctx, int src, float* H_dev) {
  if (ctx && ctx->opt.periodic) return fail(ctx, MM_ENOTSUP, "mm_compute_stray_field_fd4: periodic boundaries");
  if (!ctx || bad_mag(src) || !H_dev) return ctx ? fail(ctx, MM_EINVAL, "mm_compute_stray_field_fd4") : MM_EINVAL;
  if (ctx->opt.margin < 2) return fail(ctx, MM_ENOTSUP, "mm_compute_stray_field_fd4: needs a margin of 2 or more");
  int dims[3];
  long long lo[3];
  CKS(mm_compute_potential(ctx, src, 1, nullptr, 0, dims, lo));
  const size_t nb = (size_t)dims[0] * dims[1] * dims[2];
  CKS(ensure_buf(ctx, &ctx->fd4_C, &ctx->fd4_C_bytes, sizeof(float) * nb));
  CKS(mm_compute_potential(ctx, src, 1, ctx->fd4_C, nb, dims, lo));
  const Magnet& T = ctx->mag[1 - src];
  const int nt[3] = {T.nx, T.ny, T.nz};
  CKS(ensure_buf(ctx, &ctx->fd4_V, &ctx->fd4_V_bytes,
                 sizeof(float) * (size_t)(nt[0] + 4) * (nt[1] + 4) * (nt[2] + 4)));
  const double sigma = src == 0 ? 1.0 : -1.0;  // +1: the target is the slider
  double frac[3];
  for (int a = 0; a < 3; ++a) {
    const double su = sigma * u_cells(ctx, a, ctx->host_mech.x);
    frac[a] = su - floor(su);
  }
  CK(launch_fd4_field(ctx->fd4_C, dims, nt, ctx->opt.margin, frac, T.d, ctx->fd4_V, H_dev, ctx->st));
  return MM_OK;
}

mm_status mm_compute_stray_field_componentwise(mm_ctx* ctx, int src, float* H_dev) {
  if (ctx && ctx->opt.periodic)
    return fail(ctx, MM_ENOTSUP, "mm_compute_stray_field_componentwise: periodic boundaries");
  if (!ctx || bad_mag(src) || !H_dev)
    return ctx ? fail(ctx, MM_EINVAL, "mm_compute_stray_field_componentwise") : MM_EINVAL;
  if (!ctx->mag[0].grid || !ctx->mag[1].grid) return fail(ctx, MM_EINVAL, "grids not set");
  if (!ctx->mag[0].mat || !ctx->mag[1].mat) return fail(ctx, MM_EINVAL, "materials not set");
  CKS(replan_if_needed(ctx));
  Magnet& S = ctx->mag[src];
  const Magnet& T = ctx->mag[1 - src];
  if (!S.mset) return fail(ctx, MM_EINVAL, "magnetisation not set");
  if (S.zfft)
    return fail(ctx, MM_ENOTSUP, "mm_compute_stray_field_componentwise: sources of more than 8 layers");
  cudaStream_t st = ctx->st;
  Dir& D = S.cw;
  dir_geometry(ctx, src, true, &D);
  D.prefilter = 1;
  const int nb = D.r[2];  // every box plane
  const int P3 = 3 * S.nz, PC = 3 * nb;
  CKS(build_T(ctx, src, &D, 1));
  CKS(ensure_buf(ctx, &S.cw_Y, &S.cw_Y_bytes, sizeof(float2) * (size_t)P3 * S.kxh * S.Qy));
  CKS(ensure_buf(ctx, &D.Z3C, &D.Z3C_bytes, sizeof(float2) * (size_t)PC * S.kxh * S.Qy));
  CKS(ensure_buf(ctx, &D.YC, &D.YC_bytes, sizeof(float2) * (size_t)PC * S.kxh * D.r[1]));
  CKS(ensure_buf(ctx, &D.C, &D.C_bytes, sizeof(float) * (size_t)PC * D.r[1] * D.r[0]));
  FftTables fy;
  CKS(get_fft(ctx, S.Qy, &fy));
  CKS(join_mech(ctx));
  const float* in[2] = {ctx->mag[0].m, ctx->mag[1].m};
  const int which[1] = {src};
  int Qmax = 0;
  {
    Launch<XFwdJob> L = xfwd_launch(ctx, in, which, 1, &Qmax);
    Timer t(ctx, 0);
    CK(launch_xfwd(L, Qmax, st));
  }
  const int group = std::max(1, std::min(16, (int)((48 * 1024) / ((S.Qy + 1) * sizeof(float2)))));
  {
    Launch<YFwdJob> L{};
    L.njobs = 1;
    YFwdJob& F = L.job[0];
    F.in = S.X1; F.out = S.cw_Y; F.planes = P3; F.ny = S.ny; F.kxh = S.kxh; F.group = group; F.fy = fy;
    F.natural = 1;
    L.tile_start[1] = S.kxh * ((P3 + group - 1) / group);
    Timer t(ctx, 7);
    CK(launch_yfwd3(L, st));
  }
  {
    Launch<ZMixJob> L{};
    L.njobs = 1;
    ZMixJob& M = L.job[0];
    M.in = S.cw_Y; M.nz = S.nz; M.kxh = S.kxh; M.Qy = S.Qy; M.kyq = S.kyq;
    M.Nq = S.Nq; M.Tq = D.Tq; M.nH = 0; M.n_out = PC; M.outH = nullptr; M.outC = D.Z3C;
    M.field_nbox = nb;
    L.tile_start[1] = S.kxh * zmix_tiles(S.kyq, PC);
    Timer t(ctx, 8);
    CK(launch_zmix3(L, st));
  }
  {
    Launch<YInvJob> L{};
    L.njobs = 1;
    YInvJob& J = L.job[0];
    J.in = D.Z3C; J.natural = 1; J.planes = PC; J.kxh = S.kxh; J.group = group; J.fy = fy;
    J.is_C = 1; J.outC = D.YC;
    J.box_lo = D.box_lo[1]; J.box_len = D.box_len[1]; J.start = D.start[1]; J.r = D.r[1]; J.fir = 1;
    L.tile_start[1] = S.kxh * ((PC + group - 1) / group);
    Timer t(ctx, 9);
    CK(launch_yinv3(L, st));
  }
  {
    Launch<XInvJob> L{};
    L.njobs = 1;
    XInvJob& J = L.job[0];
    J.in = D.YC; J.out = D.C; J.planes = PC; J.rows_per_plane = D.r[1]; J.kxh = S.kxh;
    CKS(get_fft(ctx, S.Qx, &J.fx));
    J.box_lo = D.box_lo[0]; J.box_len = D.box_len[0]; J.start = D.start[0]; J.out_len = D.r[0]; J.fir = 1;
    L.tile_start[1] = (PC * D.r[1] + kRowsPerCta - 1) / kRowsPerCta;
    Timer t(ctx, 2);
    CK(launch_xinv(L, S.Qx, st));
  }
  const double sigma = src == 0 ? 1.0 : -1.0;  // +1: the target is the slider
  double frac[3];
  for (int a = 0; a < 3; ++a) {
    const double su = sigma * u_cells(ctx, a, ctx->host_mech.x);
    frac[a] = su - floor(su);
  }
  const int bdim[3] = {D.r[0], D.r[1], nb};
  const int nt[3] = {T.nx, T.ny, T.nz};
  CK(launch_field_values(D.C, bdim, nt, ctx->opt.margin, frac, H_dev, st));
  D.valid = false;
  return MM_OK;
}

// sum_j V(r_j) x S(r_i - r_j) over the magnet's own cells, scaled by s, into
// out (3 N): per component the potential path on the self box with the
// rearranged input (the result of a pass is Ms S . V', hence s / Ms).
static mm_status self_cross_S(mm_ctx* ctx, int g, const float* V, double s, float* out) {
  Magnet& M = ctx->mag[g];
  Dir& D = M.eddy;
  const float* in[2] = {ctx->mag[0].m, ctx->mag[1].m};
  in[g] = M.ed_V;
  const int which[1] = {g};
  const int what[1] = {2};
  Dir* dirs[1] = {&D};
  for (int comp = 0; comp < 3; ++comp) {
    CK(launch_cross_input(V, M.N, comp, M.ed_V, ctx->st));
    CKS(run_source_passes(ctx, in, which, 1, what, dirs));
    CK(launch_scale_into(D.C, M.N, (float)(s / M.Ms), out + comp * M.N, ctx->st));
  }
  return MM_OK;
}

mm_status mm_eddy_field(mm_ctx* ctx, int mag, const float* dBdt_dev, double sigma, float* H_dev, float* J_dev,
                        int* sweeps_out) {
  if (!ctx || bad_mag(mag) || !dBdt_dev || !(sigma >= 0) || !std::isfinite(sigma))
    return ctx ? fail(ctx, MM_EINVAL, "mm_eddy_field") : MM_EINVAL;
  if (ctx->opt.periodic) return fail(ctx, MM_ENOTSUP, "mm_eddy_field: periodic boundaries");
  CKS(prepare(ctx));
  return eddy_core(ctx, mag, dBdt_dev, sigma, H_dev, J_dev, sweeps_out);
}

mm_status mm_set_conductivity(mm_ctx* ctx, int mag, double sigma) {
  if (!ctx || bad_mag(mag) || !(sigma >= 0) || !std::isfinite(sigma))
    return ctx ? fail(ctx, MM_EINVAL, "mm_set_conductivity") : MM_EINVAL;
  if (sigma > 0 && ctx->opt.periodic) return fail(ctx, MM_ENOTSUP, "mm_set_conductivity: periodic boundaries");
  if (sigma > 0 && ctx->opt.integrator == MM_EULER)
    return fail(ctx, MM_ENOTSUP, "mm_set_conductivity: the Euler integrator (the coupling's lag is defined for RK45)");
  Magnet& M = ctx->mag[mag];
  M.sigma = sigma;
  M.B_valid = M.Heddy_valid = false;
  return MM_OK;
}

mm_status mm_eddy_field_on_other(mm_ctx* ctx, int mag, const float* J_dev, float* H_dev) {
  if (!ctx || bad_mag(mag) || !J_dev || !H_dev)
    return ctx ? fail(ctx, MM_EINVAL, "mm_eddy_field_on_other") : MM_EINVAL;
  if (ctx->opt.periodic) return fail(ctx, MM_ENOTSUP, "mm_eddy_field_on_other: periodic boundaries");
  CKS(prepare(ctx));
  return cross_eddy_field(ctx, mag, J_dev, H_dev);
}

mm_status mm_get_eddy_field(mm_ctx* ctx, int mag, float* H_dev) {
  if (!ctx || bad_mag(mag) || !H_dev) return ctx ? fail(ctx, MM_EINVAL, "mm_get_eddy_field") : MM_EINVAL;
  Magnet& M = ctx->mag[mag];
  if (!M.grid) return fail(ctx, MM_EINVAL, "grid not set");
  if (M.Heddy_valid) CK(cudaMemcpyAsync(H_dev, M.Heddy, sizeof(float) * 3 * M.N, cudaMemcpyDeviceToDevice, ctx->st));
  else CK(cudaMemsetAsync(H_dev, 0, sizeof(float) * 3 * M.nx * M.ny * M.nz, ctx->st));
  return MM_OK;
}

}  // extern "C"

// The field of the currents J (A/m^2, [3][N] of magnet g) inside the other
// magnet, at its displaced cell centres, into H ([3][N_t]).  The eddy field
// is not the gradient of a potential, so it is interpolated inside the
// moving magnet as field vectors (Sec. II): on the nodes of the potential box
// around the other magnet, (J x S)_a = the potential sum with the rearranged
// input (as self_cross_S), each component prefiltered and evaluated by the
// tricubic spline at the displaced centres (as the componentwise variant).
static mm_status cross_eddy_field(mm_ctx* ctx, int g, const float* J, float* H) {
  Magnet& S = ctx->mag[g];
  const Magnet& T = ctx->mag[1 - g];
  cudaStream_t st = ctx->st;
  Dir& D = S.eddyx;
  dir_geometry(ctx, g, true, &D);
  D.prefilter = 1;
  if (!S.zfft) CKS(build_T(ctx, g, &D));
  CKS(alloc_dir_outputs(ctx, g, &D));
  const size_t box = (size_t)D.r[0] * D.r[1] * D.r[2];
  CKS(ensure_buf(ctx, &S.ex_C3, &S.ex_bytes[0], sizeof(float) * 3 * box));
  CKS(ensure_buf(ctx, &S.ed_V, &S.ed_bytes[0], sizeof(float) * 3 * S.N));
  CKS(join_mech(ctx));
  const float* in[2] = {ctx->mag[0].m, ctx->mag[1].m};
  in[g] = S.ed_V;
  const int which[1] = {g};
  const int what[1] = {2};
  Dir* dirs[1] = {&D};
  for (int comp = 0; comp < 3; ++comp) {
    CK(launch_cross_input(J, S.N, comp, S.ed_V, st));
    CKS(run_source_passes(ctx, in, which, 1, what, dirs));
    // the path's spectra carry Ms of the source: divide it out
    CK(launch_scale_into(D.C, box, (float)(1.0 / S.Ms), S.ex_C3 + comp * box, st));
  }
  const double sigma = g == 0 ? 1.0 : -1.0;  // +1: the target is the slider
  double frac[3];
  for (int a = 0; a < 3; ++a) {
    const double su = sigma * u_cells(ctx, a, ctx->host_mech.x);
    frac[a] = su - floor(su);
  }
  const int bdim[3] = {D.r[0], D.r[1], D.r[2]};
  const int nt[3] = {T.nx, T.ny, T.nz};
  CK(launch_field_values(S.ex_C3, bdim, nt, ctx->opt.margin, frac, H, st));
  return MM_OK;
}

static mm_status eddy_core(mm_ctx* ctx, int mag, const float* dBdt_dev, double sigma, float* H_dev, float* J_dev,
                           int* sweeps_out) {
  Magnet& M = ctx->mag[mag];
  cudaStream_t st = ctx->st;
  // the box of the potential path: output nodes are the magnet's own cells
  Dir& D = M.eddy;
  const int n[3] = {M.nx, M.ny, M.nz};
  for (int a = 0; a < 3; ++a) {
    D.U0[a] = 0;
    D.box_lo[a] = -1 - ctx->opt.margin;
    D.box_len[a] = n[a] + 3 + 2 * ctx->opt.margin;
    D.start[a] = 1 + ctx->opt.margin;
    D.r[a] = n[a];
    D.guard[a] = 0;
  }
  D.full_box = false;
  D.prefilter = 0;
  if (!M.thick && (size_t)std::max(3 * M.nz, D.r[2]) * M.Qy * sizeof(float2) > 220 * 1024)
    return fail(ctx, MM_ENOTSUP, "mm_eddy_field: magnet too tall for the fused y pass");
  if (!M.zfft) CKS(build_T(ctx, mag, &D));
  const size_t N = M.N;
  const int nb = eddy_blocks(N);
  if (M.thick) CKS(ensure_buf(ctx, &D.Z3C, &D.Z3C_bytes, sizeof(float2) * (size_t)D.r[2] * M.kxh * M.Qy));
  CKS(ensure_buf(ctx, &D.YC, &D.YC_bytes, sizeof(float2) * (size_t)D.r[2] * M.kxh * D.r[1]));
  CKS(ensure_buf(ctx, &D.C, &D.C_bytes, sizeof(float) * N));
  CKS(ensure_buf(ctx, &M.ed_V, &M.ed_bytes[0], sizeof(float) * 3 * N));
  CKS(ensure_buf(ctx, &M.ed_E, &M.ed_bytes[1], sizeof(float) * 3 * N));
  CKS(ensure_buf(ctx, &M.ed_b, &M.ed_bytes[2], sizeof(double) * N));
  CKS(ensure_buf(ctx, &M.ed_phi, &M.ed_bytes[3], sizeof(double) * N));
  CKS(ensure_buf(ctx, &M.ed_J, &M.ed_bytes[4], sizeof(float) * 3 * N));
  CKS(ensure_buf(ctx, &M.ed_part, &M.ed_bytes[5], sizeof(double) * 3 * (size_t)nb));
  CKS(ensure_buf(ctx, &M.ed_stats, &M.ed_bytes[6], sizeof(double) * 4));
  CKS(join_mech(ctx));
  // 1. E_sol = -sum dB/dt x S
  CKS(self_cross_S(ctx, mag, dBdt_dev, -1.0, M.ed_E));
  // 2. phi_E: Neumann source (mean removed), red-black SOR to a residual of
  //    kTol of the source, bounded sweeps; mean of phi removed in step 3
  CK(launch_eddy_source(M.ed_E, M.nx, M.ny, M.nz, M.d, M.ed_b, M.ed_part, M.ed_stats + 3, st));
  CK(cudaMemsetAsync(M.ed_phi, 0, sizeof(double) * N, st));
  const int nmax = std::max(M.nx, std::max(M.ny, M.nz));
  const double omega = 2.0 / (1.0 + sin(3.14159265358979323846 / std::max(nmax, 2)));
  constexpr int kCheck = 25, kMaxSweeps = 40000;
  constexpr double kTol = 1e-9;
  int sweeps = 0;
  double stats[3] = {0, 0, 0};
  for (;;) {
    CK(launch_sor_residual(M.ed_phi, M.ed_b, M.ed_stats + 3, M.nx, M.ny, M.nz, M.d, M.ed_part, M.ed_stats, st));
    CK(cudaMemcpyAsync(stats, M.ed_stats, sizeof(stats), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (stats[0] <= kTol * stats[1] || stats[1] == 0.0) break;
    if (sweeps >= kMaxSweeps) {
      if (sweeps_out) *sweeps_out = sweeps;
      return fail(ctx, MM_ETIMEOUT, "mm_eddy_field: the electric potential did not converge");
    }
    CK(launch_sor_sweeps(M.ed_phi, M.ed_b, M.ed_stats + 3, M.nx, M.ny, M.nz, M.d, omega, kCheck, st));
    sweeps += kCheck;
  }
  if (sweeps_out) *sweeps_out = sweeps;
  // 3. J = sigma (E_sol - grad phi_E)
  float* J = J_dev ? J_dev : M.ed_J;
  CK(launch_eddy_current(M.ed_phi, M.ed_stats, M.ed_E, M.nx, M.ny, M.nz, M.d, sigma, J, st));
  // 4. H_eddy = sum J x S
  if (H_dev) CKS(self_cross_S(ctx, mag, J, 1.0, H_dev));
  return MM_OK;
}

extern "C" {

mm_status mm_field_div_curl(mm_ctx* ctx, const float* H_dev, int nx, int ny, int nz, double dx, double dy,
                            double dz, double* D, double* C) {
  if (!ctx) return MM_EINVAL;
  if (!H_dev || nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dy > 0) || !(dz > 0) ||
      (long long)nx * ny * nz > (1ll << 30))
    return fail(ctx, MM_EINVAL, "mm_field_div_curl: bad argument");
  const size_t cells = divcurl_cells(nx, ny, nz);
  const int nb = divcurl_blocks(nx, ny, nz);
  CKS(ensure_buf(ctx, &ctx->dc_buf, &ctx->dc_bytes, sizeof(double) * (2 * (size_t)nb + 2)));
  double out[2] = {0.0, 0.0};
  if (nb > 0) {
    CK(launch_divcurl(H_dev, nx, ny, nz, dx, dy, dz, ctx->dc_buf, ctx->dc_buf + 2 * nb, ctx->st));
    CK(cudaMemcpyAsync(out, ctx->dc_buf + 2 * nb, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  }
  if (D) *D = cells ? out[0] / (double)cells : 0.0;
  if (C) *C = cells ? out[1] / (double)cells : 0.0;
  return MM_OK;
}

mm_status mm_step(mm_ctx* ctx, int nsteps, double* t_out, double* dt_inout) {
  if (!ctx || !dt_inout || nsteps < 0) return ctx ? fail(ctx, MM_EINVAL, "mm_step") : MM_EINVAL;
  if (!(*dt_inout > 0)) return fail(ctx, MM_EINVAL, "mm_step: dt must be positive");
  CKS(prepare(ctx));
  double dt = *dt_inout;
  int done = 0;
  int guard_iter = 0;
  while (done < nsteps) {
    if (++guard_iter > 100 * (nsteps + 1) + 1000)
      return fail(ctx, MM_EINVAL, "mm_step: step size control did not converge");
    double err = 0.0;
    bool accepted = false;
    CKS(attempt_enqueue(ctx, dt));
    CKS(attempt_finish(ctx, &err));
    CKS(conclude_attempt(ctx, &dt, err, &accepted));
    if (accepted) ++done;
  }
  *dt_inout = dt;
  if (t_out) *t_out = ctx->host_mech.t;
  return MM_OK;
}

mm_status mm_step_batch(mm_ctx* const* ctxs, int npairs, int nsteps, double* t_out, double* dt_inout,
                        int* failed_pair) {
  if (failed_pair) *failed_pair = -1;
  if (npairs < 0 || nsteps < 0 || (npairs > 0 && (!ctxs || !dt_inout))) return MM_EINVAL;
  {
    std::set<const mm_ctx*> seen;
    for (int i = 0; i < npairs; ++i)
      if (!ctxs[i] || !seen.insert(ctxs[i]).second) {
        if (failed_pair) *failed_pair = i;
        return MM_EINVAL;
      }
  }
  int bad = -1;
  auto at = [&](int i, mm_status s) {
    if (s != MM_OK && bad < 0) bad = i;
    return s;
  };
#define CKB(i, expr)                     \
  do {                                   \
    mm_status s_ = at((i), (expr));      \
    if (s_ != MM_OK) {                   \
      if (failed_pair) *failed_pair = bad; \
      return s_;                         \
    }                                    \
  } while (0)
  for (int i = 0; i < npairs; ++i)
    if (!(dt_inout[i] > 0)) CKB(i, fail(ctxs[i], MM_EINVAL, "mm_step_batch: dt must be positive"));
  for (int i = 0; i < npairs; ++i) CKB(i, prepare(ctxs[i]));
  std::vector<int> done(npairs, 0), iters(npairs, 0);
  std::vector<char> active(npairs, nsteps > 0 ? 1 : 0);
  int left = nsteps > 0 ? npairs : 0;
  // every pair's first attempt is queued before the first wait; afterwards a
  // pair's next attempt is queued as soon as its previous one is concluded,
  // so the streams of the other pairs keep the GPU busy meanwhile
  for (int i = 0; i < npairs && nsteps > 0; ++i) CKB(i, attempt_enqueue(ctxs[i], dt_inout[i]));
  while (left > 0) {
    for (int i = 0; i < npairs; ++i) {
      if (!active[i]) continue;
      mm_ctx* c = ctxs[i];
      if (++iters[i] > 100 * (nsteps + 1) + 1000)
        CKB(i, fail(c, MM_EINVAL, "mm_step_batch: step size control did not converge"));
      double err = 0.0;
      bool accepted = false;
      CKB(i, attempt_finish(c, &err));
      CKB(i, conclude_attempt(c, &dt_inout[i], err, &accepted));
      if (accepted) ++done[i];
      if (done[i] < nsteps) {
        CKB(i, attempt_enqueue(c, dt_inout[i]));
      } else {
        active[i] = 0;
        --left;
      }
    }
  }
#undef CKB
  if (t_out)
    for (int i = 0; i < npairs; ++i) t_out[i] = ctxs[i]->host_mech.t;
  return MM_OK;
}

mm_status mm_fft_plan(int L, int radices[8], int* nstages) {
  if (L < 1 || !radices || !nstages) return MM_EINVAL;
  int r = L;
  for (int p : {2, 3, 5})
    while (r % p == 0) r /= p;
  if (r != 1) return MM_EINVAL;
  const std::vector<int> plan = plan_radices(L);
  if ((int)plan.size() > kMaxStages || plan.size() > 8) return MM_ENOTSUP;
  *nstages = (int)plan.size();
  for (size_t i = 0; i < plan.size(); ++i) radices[i] = plan[i];
  return MM_OK;
}

mm_status mm_assign_lanes(const double* cost, int npairs, int nlanes, int* lane_out) {
  if (npairs < 0 || nlanes < 1 || (npairs > 0 && (!cost || !lane_out))) return MM_EINVAL;
  for (int i = 0; i < npairs; ++i)
    if (!(cost[i] >= 0) || !std::isfinite(cost[i])) return MM_EINVAL;
  // longest processing time first: pairs by decreasing cost (ties by index),
  // each to the lane with the least cost so far (ties by lane index)
  std::vector<int> order(npairs);
  for (int i = 0; i < npairs; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<double> load(nlanes, 0.0);
  for (int i : order) {
    int best = 0;
    for (int l = 1; l < nlanes; ++l)
      if (load[l] < load[best]) best = l;
    lane_out[i] = best;
    load[best] += cost[i];
  }
  return MM_OK;
}

// Drops this context's tables of length L (after its work has drained), so
// the next launch builds them from the current plan of L.
static mm_status drop_fft(mm_ctx* ctx, int L) {
  auto it = ctx->ffts.find(L);
  if (it == ctx->ffts.end()) return MM_OK;
  CK(cudaStreamSynchronize(ctx->st));
  if (ctx->side) CK(cudaStreamSynchronize(ctx->side));
  cudaFree(it->second.tw_f); cudaFree(it->second.tw_d); cudaFree(it->second.pos); cudaFree(it->second.freq);
  ctx->ffts.erase(it);
  return MM_OK;
}

mm_status mm_autotune(mm_ctx* ctx, int candidates, int reps, int* n_tuned) {
  if (!ctx || candidates < 1 || candidates > 16 || reps < 1)
    return ctx ? fail(ctx, MM_EINVAL, "mm_autotune") : MM_EINVAL;
  if (n_tuned) *n_tuned = 0;
  CKS(prepare(ctx));
  // transform lengths of this context and the timing classes of the passes using them
  std::map<int, std::set<int>> classes;
  for (const Magnet& S : ctx->mag) {
    classes[S.Qx].insert(0);
    classes[S.Qx].insert(2);
    if (!S.thick) {
      classes[S.Qy].insert(1);
    } else {
      classes[S.Qy].insert(7);
      classes[S.Qy].insert(9);
    }
    if (S.zfft) classes[S.Qz].insert(8);
  }
  // the tuning runs must not disturb the caller's timing record
  const bool timing0 = ctx->timing;
  drain_timing(ctx);
  double t_ms0[kTimingClasses];
  long long t_n0[kTimingClasses];
  std::copy(ctx->t_ms, ctx->t_ms + kTimingClasses, t_ms0);
  std::copy(ctx->t_n, ctx->t_n + kTimingClasses, t_n0);
  ctx->timing = true;
  const float* in[2] = {ctx->mag[0].m, ctx->mag[1].m};
  auto run = [&]() -> mm_status {
    CKS(evaluate_fields(ctx, in, mech_params(ctx, 1, 0, 0.0, true, true)));  // warm-up
    drain_timing(ctx);
    for (int i = 0; i < kTimingClasses; ++i) {
      ctx->t_ms[i] = 0;
      ctx->t_n[i] = 0;
    }
    for (int r = 0; r < reps; ++r) CKS(evaluate_fields(ctx, in, mech_params(ctx, 1, 0, 0.0, true, true)));
    drain_timing(ctx);
    return MM_OK;
  };
  mm_status st = MM_OK;
  for (const auto& kv : classes) {
    const int L = kv.first;
    if (L <= 0) continue;
    if (tuned_plan(L, nullptr)) {  // chosen by an earlier context: use it here too
      if ((st = drop_fft(ctx, L)) != MM_OK) break;
      continue;
    }
    const auto cands = plan_candidates(L, candidates);
    if (cands.empty()) continue;
    double best_ms = 0.0;
    size_t best = 0;
    for (size_t c = 0; c < cands.size() && cands.size() > 1; ++c) {
      set_tuned_plan(L, cands[c]);
      if ((st = drop_fft(ctx, L)) != MM_OK) break;
      if ((st = run()) != MM_OK) break;
      double ms = 0.0;
      for (int cls : kv.second) ms += ctx->t_ms[cls];
      if (c == 0 || ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
    if (st != MM_OK) break;
    set_tuned_plan(L, cands[best]);
    if ((st = drop_fft(ctx, L)) != MM_OK) break;
    if (n_tuned) ++*n_tuned;
  }
  drain_timing(ctx);
  std::copy(t_ms0, t_ms0 + kTimingClasses, ctx->t_ms);
  std::copy(t_n0, t_n0 + kTimingClasses, ctx->t_n);
  ctx->timing = timing0;
  return st;
}

mm_status mm_get_tuned_plan(int L, int radices[8], int* nstages) {
  if (!radices || !nstages) return MM_EINVAL;
  std::vector<int> r;
  if (!tuned_plan(L, &r)) return MM_ESTATE;
  *nstages = (int)std::min<size_t>(8, r.size());
  for (int i = 0; i < *nstages; ++i) radices[i] = r[i];
  return MM_OK;
}

mm_status mm_get_attempt_log(mm_ctx* ctx, int capacity, double* t_out, double* dt_out, double* err_out,
                             int* accepted_out, int* n_out) {
  if (!ctx || !n_out || capacity < 0) return ctx ? fail(ctx, MM_EINVAL, "mm_get_attempt_log") : MM_EINVAL;
  const int have = (int)ctx->attempts.size();
  const int n = std::min(capacity, have);
  for (int i = 0; i < n; ++i) {
    const auto& a = ctx->attempts[(size_t)(have - n + i)];
    if (t_out) t_out[i] = a.t;
    if (dt_out) dt_out[i] = a.dt;
    if (err_out) err_out[i] = a.err;
    if (accepted_out) accepted_out[i] = a.accepted;
  }
  *n_out = n;
  return MM_OK;
}

mm_status mm_clear_attempt_log(mm_ctx* ctx) {
  if (!ctx) return MM_EINVAL;
  ctx->attempts.clear();
  return MM_OK;
}

mm_status mm_get_step_stats(mm_ctx* ctx, long long* accepted, long long* rejected) {
  if (!ctx) return MM_EINVAL;
  if (accepted) *accepted = ctx->accepted;
  if (rejected) *rejected = ctx->rejected;
  return MM_OK;
}

// Checkpoint layout: header, m of both magnets, then (when k1_valid) the
// first-same-as-last derivative k1 of both magnets, so a resumed run repeats
// the uninterrupted one bit for bit.
struct StateHeader {
  unsigned magic, version;
  unsigned long long n0, n1;
  double x, v, t, u_base[3];
  double kx1, kv1;
  int k1_valid, pad;
};

mm_status mm_get_state(mm_ctx* ctx, void* buf, size_t* bytes) {
  if (!ctx || !bytes) return MM_EINVAL;
  const size_t nm = sizeof(float) * 3 * (ctx->mag[0].N + ctx->mag[1].N);
  const size_t need = sizeof(StateHeader) + 2 * nm;
  if (!buf) {
    *bytes = need;
    return MM_OK;
  }
  if (*bytes < need) return fail(ctx, MM_ESTATE, "mm_get_state: buffer too small");
  StateHeader h{};
  h.magic = 0x4d4d5354u;
  h.version = 2u;
  h.n0 = ctx->mag[0].N;
  h.n1 = ctx->mag[1].N;
  h.x = ctx->host_mech.x; h.v = ctx->host_mech.v; h.t = ctx->host_mech.t;
  for (int a = 0; a < 3; ++a) h.u_base[a] = ctx->u_base[a];
  h.kx1 = ctx->host_mech.kx[0];
  h.kv1 = ctx->host_mech.kv[0];
  h.k1_valid = ctx->k1_valid ? 1 : 0;
  memcpy(buf, &h, sizeof(h));
  char* p = (char*)buf + sizeof(h);
  for (int g = 0; g < 2; ++g) {
    if (ctx->mag[g].N) CK(cudaMemcpyAsync(p, ctx->mag[g].m, sizeof(float) * 3 * ctx->mag[g].N,
                                          cudaMemcpyDeviceToHost, ctx->st));
    p += sizeof(float) * 3 * ctx->mag[g].N;
  }
  for (int g = 0; g < 2; ++g) {
    if (ctx->mag[g].N && ctx->k1_valid)
      CK(cudaMemcpyAsync(p, ctx->mag[g].k[0], sizeof(float) * 3 * ctx->mag[g].N, cudaMemcpyDeviceToHost,
                         ctx->st));
    else
      memset(p, 0, sizeof(float) * 3 * ctx->mag[g].N);
    p += sizeof(float) * 3 * ctx->mag[g].N;
  }
  CK(cudaStreamSynchronize(ctx->st));
  *bytes = need;
  return MM_OK;
}

mm_status mm_set_state(mm_ctx* ctx, const void* buf, size_t bytes) {
  if (ctx) reset_eddy(ctx);
  if (!ctx || !buf) return MM_EINVAL;
  if (bytes < sizeof(StateHeader)) return fail(ctx, MM_ESTATE, "mm_set_state: short buffer");
  StateHeader h;
  memcpy(&h, buf, sizeof(h));
  if (h.magic != 0x4d4d5354u || h.version != 2u || h.n0 != ctx->mag[0].N || h.n1 != ctx->mag[1].N)
    return fail(ctx, MM_ESTATE, "mm_set_state: header does not match this context");
  const size_t nm = sizeof(float) * 3 * (h.n0 + h.n1);
  if (bytes < sizeof(StateHeader) + 2 * nm) return fail(ctx, MM_ESTATE, "mm_set_state: short buffer");
  const char* p = (const char*)buf + sizeof(h);
  for (int g = 0; g < 2; ++g) {
    CK(cudaMemcpyAsync(ctx->mag[g].m, p, sizeof(float) * 3 * ctx->mag[g].N, cudaMemcpyHostToDevice, ctx->st));
    p += sizeof(float) * 3 * ctx->mag[g].N;
    ctx->mag[g].mset = true;
  }
  if (h.k1_valid)
    for (int g = 0; g < 2; ++g) {
      CK(cudaMemcpyAsync(ctx->mag[g].k[0], p, sizeof(float) * 3 * ctx->mag[g].N, cudaMemcpyHostToDevice,
                         ctx->st));
      p += sizeof(float) * 3 * ctx->mag[g].N;
    }
  CK(cudaStreamSynchronize(ctx->st));
  for (int a = 0; a < 3; ++a) ctx->u_base[a] = h.u_base[a];
  ctx->host_mech.x = h.x; ctx->host_mech.v = h.v; ctx->host_mech.t = h.t;
  ctx->host_mech.kx[0] = h.kx1;
  ctx->host_mech.kv[0] = h.kv1;
  ctx->k1_valid = false;
  if (ctx->planned) CKS(replan_if_needed(ctx));
  if (h.k1_valid) {
    CKS(upload_mech(ctx));  // carries kx[0], kv[0]
    ctx->k1_valid = true;
  }
  return MM_OK;
}

mm_status mm_eval_kernel_fp64(int kind, int n, const double* offsets_dev, double dx, double dy, double dz,
                              double* out_dev) {
  if ((kind != 0 && kind != 1) || n < 0 || !offsets_dev || !out_dev || !(dx > 0) || !(dy > 0) || !(dz > 0))
    return MM_EINVAL;
  cudaError_t e = eval_points_fp64(kind, n, offsets_dev, dx, dy, dz, out_dev, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e == cudaSuccess ? MM_OK : MM_ECUDA;
}

mm_status mm_get_plan_info(mm_ctx* ctx, int src, int fft_dims[3], int box_dims[3], long long box_lo[3],
                           int coef_dims[3]) {
  if (!ctx || bad_mag(src)) return MM_EINVAL;
  if (!ctx->planned) CKS(ensure_plan(ctx));
  const Magnet& S = ctx->mag[src];
  if (fft_dims) { fft_dims[0] = S.Qx; fft_dims[1] = S.Qy; fft_dims[2] = S.zfft ? S.Qz : 0; }
  for (int a = 0; a < 3; ++a) {
    if (box_dims) box_dims[a] = S.dir.box_len[a];
    if (box_lo) box_lo[a] = S.dir.box_lo[a];
    if (coef_dims) coef_dims[a] = S.dir.r[a];
  }
  return MM_OK;
}

mm_status mm_set_timing(mm_ctx* ctx, int on) {
  if (!ctx) return MM_EINVAL;
  ctx->timing = on != 0;
  return MM_OK;
}

mm_status mm_get_timing(mm_ctx* ctx, int cls, double* total_ms, long long* launches) {
  if (!ctx || cls < 0 || cls >= kTimingClasses) return MM_EINVAL;
  drain_timing(ctx);
  if (total_ms) *total_ms = ctx->t_ms[cls];
  if (launches) *launches = ctx->t_n[cls];
  return MM_OK;
}

mm_status mm_reset_timing(mm_ctx* ctx) {
  if (!ctx) return MM_EINVAL;
  drain_timing(ctx);
  for (int i = 0; i < kTimingClasses; ++i) { ctx->t_ms[i] = 0; ctx->t_n[i] = 0; }
  return MM_OK;
}

long long mm_launch_count(const mm_ctx* ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"
