// C ABI and host orchestration of the rotating-shell library (see rsc.h).
//
// One context = one problem (parameters + truncation) on one CUDA stream.
// A time step (Eq. discrete) and a Jacobian action (Secs. 3.3-3.4) are a
// fixed sequence of kernel launches on that stream; Newton-GMRES (Eq.
// precond, Eq. twNewton) drives them from the host with one small
// device-to-host read per GMRES iteration for the Hessenberg column.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <cstdint>
#include <memory>
#include <mutex>
#include <thread>
#include <type_traits>
#include <vector>

#include "kernels.cuh"
#include "chain_async.cuh"
#include "legendre_tc.cuh"
#include "legendre_tc_analysis.cuh"
#include "krylov_split.cuh"
#include "chain_df.cuh"
#include "chain_cr.cuh"
#include "products_lin.cuh"
#include "radial_rhs_f32.cuh"
#include "cr_factor_gpu.cuh"
#include "factor_gpu.cuh"
#include "rsc_internal.h"

using namespace rsc;

namespace {

constexpr int kMaxKrylov = 2048;
constexpr int kMaxChainParts = 4;   // parts per chain of the partitioned double-float solve

struct DevFactor {
  double dt = std::nan("");
  long* chain_off = nullptr;
  double2* G = nullptr;
  double2* H = nullptr;
  double2* W = nullptr;
  double* Tinv = nullptr;
  // double-float copies of G, H, W (mixed-precision contexts): float4 {re_hi, im_hi, re_lo, im_lo}
  float4* Gs = nullptr;
  float4* Hs = nullptr;
  float4* Ws = nullptr;
  // partitioned chains of the double-float solve (chain_parts > 1; HostFactor): part table,
  // spikes, reduced inverses and their index tables, and the reduced solution z
  int npart = 0, nz = 0, nu_max = 0;
  long* parts = nullptr;
  float4* Vsp = nullptr;
  float4* Wsp = nullptr;
  float4* red = nullptr;
  long* red_off = nullptr;
  int* red_nu = nullptr;
  int* zoff = nullptr;
  long* unk_row = nullptr;
  int* blk_z = nullptr;
  double2* zbuf = nullptr;
  // odd-even reduced chains of the double-float solve (chain_cr; HostFactorCR): inverses of
  // the odd diagonal blocks and the twisted factors of the reduced chains, float4 pairs
  long* cr_odd_off = nullptr;
  long* cr_red_off = nullptr;
  float4* Ds = nullptr;
  float4* Gr = nullptr;
  float4* Hr = nullptr;
  float4* Wr = nullptr;
  double cr_s = 0.0;   // wall time of their factorisation (s)
  int cr_on_gpu = 0;   // where it ran
  bool valid = false;
};

template <typename R>
struct LegDev {
  R* buf[8] = {nullptr};  // P dP Ps Pw dPw Psw twc tws
  DevLegendre<R> view() const {
    return DevLegendre<R>{buf[0], buf[1], buf[2], buf[3], buf[4], buf[5], buf[6], buf[7]};
  }
};

struct FactorShare;

}  // namespace

struct rsc_ctx {
  rsc_params p{};
  Dims d;
  HostTables t;
  cudaStream_t s = nullptr;
  int device = 0;
  // geometry
  int *d_m_of = nullptr, *d_pstart = nullptr, *d_pair_l = nullptr, *d_pair_m = nullptr;
  long* d_leg_off = nullptr;
  double *d_rc = nullptr, *d_rd = nullptr, *d_EcT0 = nullptr, *d_EcT2 = nullptr;
  double* d_EcT1 = nullptr;
  double *d_EdT0 = nullptr, *d_EdT1 = nullptr, *d_EdT2 = nullptr, *d_R0T = nullptr, *d_R1T = nullptr;
  float *f_EdT0 = nullptr, *f_EdT1 = nullptr, *f_EdT2 = nullptr, *f_R0T = nullptr, *f_R1T = nullptr;
  float* f_rd = nullptr;
  float *f_EcT0 = nullptr, *f_EcT2 = nullptr;
  LegDev<double> leg64;
  LegDev<float> leg32;
  // workspace (sized for FP64; the FP32 path uses the front part)
  void *SR = nullptr, *FC = nullptr, *FCU = nullptr, *FA = nullptr, *AR = nullptr;
  void* AR0 = nullptr;   // analysed products of x^n during a second-order step
  void* UG = nullptr;    // grid values of the cached base state, [9][Nd][nlat][nphi]
  int ug_prec = 0;       // precision UG holds for the current FCU: 0 none, 1 FP64, 2 FP32
  double2* rhs = nullptr;
  double2* mid = nullptr;   // chain sweep staging, [2 nm][3][Nr]
  double* xtmp = nullptr;
  double* vtmp = nullptr;
  double* rtmp = nullptr;
  double* ustate = nullptr;   // device copy of the state of the *_host calls
  double* d_Ef[4] = {nullptr, nullptr, nullptr, nullptr};   // E0, E1, E2, E4 row-major [j][k]
  int factor_gpu = 1;          // 1: factorise on the GPU (k_factor_*), 0: on the host
  int refine = 1;              // iterative-refinement steps of every FP64 e/f chain solve
  double* ref_tmp = nullptr;   // correction of a refinement step
  double factor_s = 0.0;       // wall time of the last factorisation (s)
  int factor_on_gpu = 0;       // where the last factorisation ran
  double factor_cr_s = 0.0;    // the same for the last factorisation of the reduced chains
  int factor_cr_on_gpu = 0;
  // factorisations, two slots (time stepping dt and Newton dt)
  DevFactor fac[2];
  int fac_next = 0;
  // factorisations shared with the other instances of a batch that have the same operator
  // (truncation, Ek, Pr, eta, precision, Coriolis treatment); null for a lone context
  std::shared_ptr<FactorShare> share;
  // Krylov
  double* V = nullptr;
  float2* Vs = nullptr;   // the same basis as (hi, lo) float pairs (krylov_split)
  int V_cols = 0;
  long ldV = 0;   // column stride of V and Vs
  int krylov_split = 1;   // 1: orthogonalise against Vs in double-float arithmetic
  double* partial = nullptr;
  double* dots = nullptr;
  double* h_pinned = nullptr;
  int nblk_dot = 0;
  int cluster = 8;  // CTAs per chain in the cluster chain solve
  int chain_async = 0;   // 1: sweeps with column-split warps and st.async / mbarrier exchange
  int chain_df = 0;       // mixed path: 2 / 4 = double-float chain solve with that many warps
                          // per row group (chain_df.cuh), 0 = the FP64 kernels
  int cluster_df = 8;     // CTAs per cluster of the double-float sweeps
  int chain_parts = 1;    // parts per chain of the double-float solve (1: unpartitioned)
  int chain_cr = 0;       // 1: the double-float solve on odd-even reduced chains (chain_cr.cuh)
  int* d_cr_pairs = nullptr;   // pairs with odd l - m (n_cr_odd), then even (n_cr_even)
  int n_cr_odd = 0, n_cr_even = 0;
  float4* d_E01 = nullptr;     // [j][k] {E0 hi, E0 lo, E1 hi, E1 lo} at the collocation radii
  float4* d_cr_rowf = nullptr;    // [j] {2 / r^3 hi, lo, 2 / r^2 hi, lo}
  float4* d_cr_pairf = nullptr;   // [p][2] {a l, a}, {c (l + 1), c} (coupling coefficients)
  float4* cr_w = nullptr;      // E0 u, E1 u of the odd blocks, [2][2 P Nr]
  // second stream: the temperature solve runs beside the e/f chain solve
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int rt_synth[2] = {1, 1}, rt_anal[2] = {1, 1};  // radii per block, [fp64, fp32]
  int radial_f32_grid = 0, rhs_lin_grid = 0;     // persistent FP32 radial kernels (0: not used)
  int wpb[2] = {0, 0};     // warps per block of the products kernel (0: largest that fits)
  int ppb[2] = {0, 0};     // pairs per block of the right-hand-side kernel (0: 256 / Nr)
  int atc[2] = {16, 16};   // latitudes per staged chunk of the analysis tables
  int lpw[2] = {1, 1};     // latitudes per warp of the products kernel
  int anal_tc = 0;         // 1: tensor-core Legendre analysis on the mixed path
  float* ta_tiles = nullptr;   // its A tiles (hi | lo per (m, parity, table, chunk))
  long* ta_off = nullptr;
  int ta_nchunk = 0;
  double tune_ms[6] = {0, 0, 0, 0, 0, 0};
  // tensor-core Legendre synthesis (FP32 path): A tiles, offsets, padded K, status word
  float* tc_tiles = nullptr;
  long* tc_off = nullptr;
  int* tc_kpad = nullptr;
  int tc_nmt = 1;
  int tc_kmax = 0;          // largest padded K of the synthesis tiles
  int synth_pipe = 0;       // 1: two-stage tensor-core synthesis (where it fits)
  int* d_status = nullptr;
  // tracing: launch counter, per-kernel CUDA-event timing and algorithmic traffic
  long launches = 0;
  bool prof_on = false;
  unsigned prof_mask = 0;      // kernel ids whose launches are bracketed by events
  // CUDA graph of one Jacobian action (replayed inside GMRES)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t jvp_exec = nullptr;
  long jvp_nodes = 0;
  struct { int fp32; const double* U; double C; long J; double dt; } jvp_key{};
  const double** d_slots = nullptr;   // [u, out] of the replayed action
  double* d_cslot = nullptr;          // c = u_J of the replayed action
  double* jvp_y = nullptr;            // solve output of the replayed action
  // diagnostics: Gauss-Legendre radial rule and Chebyshev tables (built on first use)
  int ke_nq = 0;
  double *d_keT = nullptr, *d_kedT = nullptr, *d_ker = nullptr, *d_kew = nullptr;
  double* d_diag = nullptr;   // [KE, Nu_in, Nu_out]
  // Ra continuation: the last three converged states, the conductive state, argmax scratch
  double* cont_hist = nullptr;
  double* cont_cond = nullptr;
  double* amax_v = nullptr;
  long* amax_i = nullptr;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  double prof_ms[RSC_NUM_KERNELS] = {0};
  long prof_launches[RSC_NUM_KERNELS] = {0};
  double prof_bytes[RSC_NUM_KERNELS] = {0};
  double prof_flops[RSC_NUM_KERNELS] = {0};
  std::string err;
  DevGeom geom() const {
    DevGeom g;
    g.L = d.L; g.Ms = d.Ms; g.Nr = d.Nr; g.Nd = d.Nd; g.nlat = d.nlat; g.nlat2 = d.nlat2;
    g.nphi = d.nphi; g.nm = d.nm; g.K = d.K; g.P = d.P; g.r_in = d.r_in; g.r_out = d.r_out;
    g.m_of = d_m_of; g.pstart = d_pstart; g.leg_off = d_leg_off; g.pair_l = d_pair_l;
    g.pair_m = d_pair_m; g.rc = d_rc; g.rd = d_rd; g.EcT0 = d_EcT0; g.EcT2 = d_EcT2;
    g.EcT1 = d_EcT1;
    g.EdT0 = d_EdT0; g.EdT1 = d_EdT1; g.EdT2 = d_EdT2; g.R0T = d_R0T; g.R1T = d_R1T;
    g.EdT0f = f_EdT0; g.EdT1f = f_EdT1; g.EdT2f = f_EdT2; g.R0Tf = f_R0T; g.R1Tf = f_R1T;
    g.rdf = f_rd;
    g.EcT0f = f_EcT0;
    g.EcT2f = f_EcT2;
    return g;
  }
};

namespace {

template <typename R> const LegDev<R>& leg(const rsc_ctx* ctx);
template <> const LegDev<double>& leg<double>(const rsc_ctx* ctx) { return ctx->leg64; }
template <> const LegDev<float>& leg<float>(const rsc_ctx* ctx) { return ctx->leg32; }

#define CK(call)                                                              \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
      return RSC_ECUDA;                                                       \
    }                                                                         \
  } while (0)

#define CKS(expr)                                                             \
  do {                                                                        \
    rsc_status s_ = (expr);                                                   \
    if (s_ != RSC_OK) return s_;                                              \
  } while (0)

int round32(int v) { return ((v + 31) / 32) * 32; }

cudaEvent_t take_event(rsc_ctx* ctx) {
  if (!ctx->ev_pool.empty()) {
    cudaEvent_t e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one kernel launch: counts it, adds its algorithmic bytes / flops
// and, when tracing is on, records CUDA events around it on the context stream.
struct KSpan {
  rsc_ctx* ctx;
  int id;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  KSpan(rsc_ctx* c, int kid, double bytes, double flops) : ctx(c), id(kid) {
    ctx->launches++;
    if (ctx->prof_on && ((ctx->prof_mask >> id) & 1u)) {
      ctx->prof_launches[id]++;
      ctx->prof_bytes[id] += bytes;
      ctx->prof_flops[id] += flops;
      e0 = take_event(ctx);
      e1 = take_event(ctx);
      cudaEventRecord(e0, ctx->s);
    }
  }
  ~KSpan() {
    if (e0) {
      cudaEventRecord(e1, ctx->s);
      ctx->ev_pending.push_back({id, {e0, e1}});
    }
  }
};

void drain_events(rsc_ctx* ctx) {
  if (ctx->ev_pending.empty()) return;
  cudaStreamSynchronize(ctx->s);
  for (auto& pe : ctx->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess)
      ctx->prof_ms[pe.first] += ms;
    ctx->ev_pool.push_back(pe.second.first);
    ctx->ev_pool.push_back(pe.second.second);
  }
  ctx->ev_pending.clear();
}

template <typename T>
rsc_status upload(rsc_ctx* ctx, T** dst, const T* src, size_t count) {
  CK(cudaMalloc((void**)dst, std::max<size_t>(1, count) * sizeof(T)));
  if (count) CK(cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
  return RSC_OK;
}

std::vector<double> transpose(const std::vector<double>& a, int rows, int cols) {
  std::vector<double> o((size_t)rows * cols);
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) o[(size_t)c * rows + r] = a[(size_t)r * cols + c];
  return o;
}

rsc_status check_params(const rsc_params* p) {
  if (!p) return RSC_EINVAL;
  if (p->L < 1 || p->L > 255 || p->Ms < 1 || p->Ms > p->L || p->Nr < 6 || p->Nr > 128)
    return RSC_EINVAL;
  if (!(p->eta > 0 && p->eta < 1) || !(p->Ek > 0) || !(p->Pr > 0) || !std::isfinite(p->Ra))
    return RSC_EINVAL;
  if (p->precision != RSC_FP64 && p->precision != RSC_MIXED) return RSC_EINVAL;
  if (p->explicit_coriolis != 0 && p->explicit_coriolis != 1) return RSC_EINVAL;
  return RSC_OK;
}

void free_factor(DevFactor& f) {
  cudaFree(f.chain_off);
  cudaFree(f.G);
  cudaFree(f.H);
  cudaFree(f.W);
  cudaFree(f.Tinv);
  cudaFree(f.Gs);
  cudaFree(f.Hs);
  cudaFree(f.Ws);
  void* extra[] = {f.parts, f.Vsp, f.Wsp, f.red, f.red_off, f.red_nu, f.zoff, f.unk_row, f.blk_z,
                   f.zbuf, f.cr_odd_off, f.cr_red_off, f.Ds, f.Gr, f.Hr, f.Wr};
  for (void* b : extra) cudaFree(b);
  f = DevFactor();
}

// Factorisations of one operator shared by several contexts (the instances of a batch with
// the same truncation, Ek, Pr, eta, precision and Coriolis treatment; Sec. 3.2: the factors
// depend on (Ek, dt) and the truncation only, not on Ra).  One slot per dt, built by the
// first context that needs it and kept until the last sharing context is destroyed.
struct FactorShare {
  static constexpr int kMaxSlots = 4;
  std::mutex mu;
  std::vector<DevFactor*> slots;
  ~FactorShare() {
    for (DevFactor* f : slots) {
      free_factor(*f);
      delete f;
    }
  }
};

template <typename R>
rsc_status upload_legendre(rsc_ctx* ctx, LegDev<R>& L) {
  const HostTables& t = ctx->t;
  const std::vector<double>* src[6] = {&t.P, &t.dP, &t.Ps, &t.Pw, &t.dPw, &t.Psw};
  for (int q = 0; q < 6; ++q) {
    std::vector<R> v(src[q]->begin(), src[q]->end());
    CKS(upload(ctx, &L.buf[q], v.data(), v.size()));
  }
  const int K1 = ctx->d.K + 1, nphi = ctx->d.nphi;
  std::vector<R> c((size_t)K1 * nphi), s((size_t)K1 * nphi);
  for (int a = 0; a < K1; ++a)
    for (int j = 0; j < nphi; ++j) {
      // exact reduction of the angle to [0, nphi) before the trig call
      const long q = ((long)a * j) % nphi;
      const double ang = 2.0 * 3.14159265358979323846 * (double)q / nphi;
      c[(size_t)a * nphi + j] = (R)std::cos(ang);
      s[(size_t)a * nphi + j] = (R)std::sin(ang);
    }
  CKS(upload(ctx, &L.buf[6], c.data(), c.size()));
  CKS(upload(ctx, &L.buf[7], s.data(), s.size()));
  return RSC_OK;
}

// A tiles of the tensor-core synthesis: for each (m, parity s, table w, latitude tile),
// 128 latitudes x Kpad degrees of the class in the K-major core-matrix layout,
// TF32 hi part then lo part.
// The two-stage tensor-core synthesis fits in the opt-in shared memory of a CTA.
bool synth_pipe_fits(int kmax) { return kmax > 0 && tc_synth_smem(kmax, true) <= 227 * 1024; }

rsc_status build_tc_tables(rsc_ctx* ctx) {
  const Dims& d = ctx->d;
  const HostTables& t = ctx->t;
  const int nmt = (d.nlat2 + 127) / 128;
  std::vector<int> kpad(d.nm);
  std::vector<long> off((size_t)d.nm * 2 * 3 * nmt);
  long total = 0;
  for (int a = 0; a < d.nm; ++a) {
    const int nl = d.L - t.m_of[a] + 1;
    kpad[a] = (((nl + 1) / 2) + 7) / 8 * 8;
    for (int q = 0; q < 2 * 3 * nmt; ++q) {
      off[(size_t)a * 2 * 3 * nmt + q] = total;
      total += 2L * 128 * kpad[a];
    }
  }
  std::vector<float> tiles((size_t)total, 0.0f);
  const std::vector<double>* tab[3] = {&t.P, &t.dP, &t.Ps};
  for (int a = 0; a < d.nm; ++a) {
    const int nl = d.L - t.m_of[a] + 1;
    const int Kp = kpad[a];
    for (int s = 0; s < 2; ++s)
      for (int w = 0; w < 3; ++w)
        for (int mt = 0; mt < nmt; ++mt) {
          float* hi = &tiles[(size_t)off[((size_t)(a * 2 + s) * 3 + w) * nmt + mt]];
          float* lo = hi + 128 * Kp;
          for (int row = 0; row < 128; ++row)
            for (int k = 0; k < Kp; ++k) {
              const int th = mt * 128 + row;
              const int q = s + 2 * k;
              float v = 0.0f;
              if (th < d.nlat2 && q < nl) v = (float)(*tab[w])[t.leg_off[a] + (size_t)q * d.nlat2 + th];
              uint32_t bits;
              std::memcpy(&bits, &v, 4);
              bits &= 0xFFFFE000u;
              float h;
              std::memcpy(&h, &bits, 4);
              const size_t o = (size_t)(row >> 3) * (Kp / 4) * 32 + (size_t)(k >> 2) * 32 + (row & 7) * 4 + (k & 3);
              hi[o] = h;
              lo[o] = v - h;
            }
        }
  }
  CKS(upload(ctx, &ctx->tc_tiles, tiles.data(), tiles.size()));
  CKS(upload(ctx, &ctx->tc_off, off.data(), off.size()));
  CKS(upload(ctx, &ctx->tc_kpad, kpad.data(), kpad.size()));
  ctx->tc_nmt = nmt;
  int kmax = 0;
  for (int k : kpad) kmax = std::max(kmax, k);
  ctx->tc_kmax = kmax;
  ctx->synth_pipe = synth_pipe_fits(kmax) ? 1 : 0;
  return RSC_OK;
}

// A tiles of the tensor-core analysis: per (m, parity s, table w in {P, P/sin, dP/dtheta},
// latitude chunk c) a 128 x kTaKc tile, rows = degrees l = m + s + 2 row, columns = north
// latitudes c kTaKc + k, weights folded (the analysis tables), TF32 hi and lo parts in the
// K-major core-matrix layout of the synthesis tiles.
rsc_status build_ta_tables(rsc_ctx* ctx) {
  const Dims& d = ctx->d;
  const HostTables& t = ctx->t;
  const int nchunk = (d.nlat2 + kTaKc - 1) / kTaKc;
  std::vector<long> off((size_t)d.nm * 2 * 3 * nchunk);
  const long tile = 2L * 128 * kTaKc;
  for (size_t q = 0; q < off.size(); ++q) off[q] = (long)q * tile;
  std::vector<float> tiles(off.size() * (size_t)tile, 0.0f);
  const std::vector<double>* tab[3] = {&t.Pw, &t.Psw, &t.dPw};
  for (int a = 0; a < d.nm; ++a) {
    const int nl = d.L - t.m_of[a] + 1;
    for (int sp = 0; sp < 2; ++sp)
      for (int w = 0; w < 3; ++w)
        for (int c = 0; c < nchunk; ++c) {
          float* hi = &tiles[(size_t)off[((size_t)(a * 2 + sp) * 3 + w) * nchunk + c]];
          float* lo = hi + 128 * kTaKc;
          for (int row = 0; row < 128; ++row)
            for (int k = 0; k < kTaKc; ++k) {
              const int th = c * kTaKc + k;
              const int q = sp + 2 * row;
              float v = 0.0f;
              if (th < d.nlat2 && q < nl) v = (float)(*tab[w])[t.leg_off[a] + (size_t)th * nl + q];
              uint32_t bits;
              std::memcpy(&bits, &v, 4);
              bits &= 0xFFFFE000u;
              float h;
              std::memcpy(&h, &bits, 4);
              const size_t o = (size_t)(row >> 3) * (kTaKc / 4) * 32 + (size_t)(k >> 2) * 32 +
                               (row & 7) * 4 + (k & 3);
              hi[o] = h;
              lo[o] = v - h;
            }
        }
  }
  CKS(upload(ctx, &ctx->ta_tiles, tiles.data(), tiles.size()));
  CKS(upload(ctx, &ctx->ta_off, off.data(), off.size()));
  ctx->ta_nchunk = nchunk;
  return RSC_OK;
}

// Whether `threads` threads of `fn` fit the register file and the block size limit.
bool threads_fit(const void* fn, int threads) {
  cudaFuncAttributes at{};
  if (cudaFuncGetAttributes(&at, fn) != cudaSuccess) return false;
  return threads <= 1024 && (long)threads * std::max(at.numRegs, 1) <= 65536 &&
         threads <= at.maxThreadsPerBlock;
}

// Radial sizes with a compile-time instantiation of the FP32 radial kernels: 1 for
// (N_r, N_d) = (64, 96), 2 for (96, 144), else 0 (sizes read at run time).
int radial_fixed(const Dims& d) {
  return (d.Nr == 64 && d.Nd == 96) ? 1 : (d.Nr == 96 && d.Nd == 144) ? 2 : 0;
}

rsc_status set_smem_limits(rsc_ctx* ctx) {
  const int big = 200 * 1024;
  CK(cudaFuncSetAttribute(k_products<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(k_products<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(k_products<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(k_products<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(k_radial<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(k_radial<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  {
    // the persistent FP32 radial kernels: one or two blocks per SM with the tables staged
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const Dims& d = ctx->d;
    const size_t lim = 227 * 1024;
    // The attribute belongs to the kernel on this device, not to this context: it only ever
    // grows (the largest need of any context so far), so that a context of smaller sizes
    // created later never lowers it under an earlier one.
    struct AttrSet {
      const void* fn;
      int dev;
      size_t smem;
    };
    static std::mutex attr_mu;
    static std::vector<AttrSet> attr_set;
    auto grid_for = [&](const void* fn, int thr, size_t smem, bool fits) -> int {
      if (!fits || thr > 1024 || smem > lim) return 0;
      {
        std::lock_guard<std::mutex> lk(attr_mu);
        size_t* have = nullptr;
        for (auto& e : attr_set)
          if (e.fn == fn && e.dev == dev) have = &e.smem;
        if (!have) {
          attr_set.push_back(AttrSet{fn, dev, 0});
          have = &attr_set.back().smem;
        }
        if (smem > *have) {
          if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return 0;
          *have = smem;
        }
      }
      int nb = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, thr, smem) != cudaSuccess || nb < 1)
        return 0;
      return (int)std::min<long>((long)nb * nsm, d.P);
    };
    const int tr = 4 * ((d.Nd + 7) / 8 * 8), th = 4 * ((d.Nr + 7) / 8 * 8);
    const int fix = radial_fixed(d);
    const void* fr = fix == 1 ? (const void*)k_radial_f32<64, 96>
                   : fix == 2 ? (const void*)k_radial_f32<96, 144> : (const void*)k_radial_f32<0, 0>;
    const void* fh = fix == 1 ? (const void*)k_rhs_lin<64, 96>
                   : fix == 2 ? (const void*)k_rhs_lin<96, 144> : (const void*)k_rhs_lin<0, 0>;
    ctx->radial_f32_grid = grid_for(fr, tr, radial_f32_smem(d.Nr, d.Nd), tr >= 3 * d.Nr);
    ctx->rhs_lin_grid = grid_for(fh, th, rhs_lin_smem(d.Nr, d.Nd),
                                 th <= 512 && th >= 3 * d.Nr && 2 * th >= 4 * d.Nd);
    cudaGetLastError();   // a refused attribute leaves the kernels unused, not an error
  }
  // radii per block of the Legendre kernels: as many as the register file allows (<= 4)
  auto rt_for = [&](const void* fn, int threads_x) {
    cudaFuncAttributes at{};
    if (cudaFuncGetAttributes(&at, fn) != cudaSuccess) return 1;
    int rt = 4;
    while (rt > 1 && ((long)rt * threads_x * std::max(at.numRegs, 1) > 65536 || rt * threads_x > 1024))
      --rt;
    return rt;
  };
  ctx->rt_synth[0] = rt_for((const void*)k_synth<double>, round32(ctx->d.nlat2));
  ctx->rt_synth[1] = rt_for((const void*)k_synth<float>, round32(ctx->d.nlat2));
  ctx->rt_anal[0] = rt_for((const void*)k_analysis<double>, round32(ctx->d.L + 1));
  ctx->rt_anal[1] = rt_for((const void*)k_analysis<float>, round32(ctx->d.L + 1));
  // pairs per block of the right-hand side: 256 / Nr, halved until the registers fit
  for (int p = 0; p < 2; ++p) {
    int q = std::max(1, 256 / round32(ctx->d.Nr));
    const void* fn = p ? (const void*)k_rhs<float> : (const void*)k_rhs<double>;
    while (q > 1 && !threads_fit(fn, round32(ctx->d.Nr) * q)) q /= 2;
    ctx->ppb[p] = q;
  }
  CK(cudaFuncSetAttribute(k_synth<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(k_synth<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(k_analysis<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(k_analysis<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(k_rhs<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(k_rhs<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(k_synth_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 226 * 1024));
  CK(cudaFuncSetAttribute(k_synth_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 226 * 1024));
  CK(cudaFuncSetAttribute(k_analysis_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ta_smem()));
  CK(cudaFuncSetAttribute(k_dots_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * (kMaxKrylov + 2) * 8));
  return RSC_OK;
}

// Whether the factorisation runs on the device: the GPU kernels hold one block of up to
// kFacMaxNr rows in shared memory and build unpartitioned chains (the spikes of partitioned
// chains come from the host routine).
bool factor_on_device(const rsc_ctx* ctx) {
  return ctx->factor_gpu && ctx->d.Nr <= kFacMaxNr && ctx->chain_parts == 1;
}

// The factors of one dt on the device (factor_gpu.cuh), FP64, and their double-float
// copies on a mixed-precision context.
rsc_status gpu_factor(rsc_ctx* ctx, double dt, DevFactor& f) {
  const Dims& d = ctx->d;
  const int nchains = 2 * d.nm;
  std::vector<long> off(nchains + 1);
  long o = 0;
  for (int c = 0; c < nchains; ++c) {
    off[c] = o;
    o += d.L - ctx->t.m_of[c / 2] + 1;
  }
  off[nchains] = o;
  const size_t blk = (size_t)d.Nr * d.Nr;
  const size_t nent = (size_t)o * blk;
  CKS(upload(ctx, &f.chain_off, off.data(), off.size()));
  CK(cudaMalloc(&f.G, nent * sizeof(double2)));
  CK(cudaMalloc(&f.H, nent * sizeof(double2)));
  CK(cudaMalloc(&f.W, nent * sizeof(double2)));
  CK(cudaMalloc(&f.Tinv, (size_t)(d.L + 1) * blk * sizeof(double)));
  CK(cudaMemsetAsync(f.H, 0, nent * sizeof(double2), ctx->s));   // H of the end blocks stays 0
  CK(cudaMemsetAsync(f.W, 0, nent * sizeof(double2), ctx->s));
  int* status = nullptr;
  CK(cudaMalloc(&status, (nchains + 1) * sizeof(int)));
  CK(cudaMemsetAsync(status, 0, (nchains + 1) * sizeof(int), ctx->s));
  FacGeom g;
  g.Nr = d.Nr;
  g.L = d.L;
  g.nm = d.nm;
  g.m_of = ctx->d_m_of;
  g.chain_off = f.chain_off;
  g.rc = ctx->d_rc;
  g.E0 = ctx->d_Ef[0];
  g.E1 = ctx->d_Ef[1];
  g.E2 = ctx->d_Ef[2];
  g.E4 = ctx->d_Ef[3];
  g.Ek = ctx->p.Ek;
  g.Pr = ctx->p.Pr;
  g.inv_dt = std::isfinite(dt) ? 1.0 / dt : 0.0;
  g.explicit_coriolis = ctx->p.explicit_coriolis ? 1 : 0;
  const size_t smem = fac_smem_bytes(d.Nr);
  for (const void* fn : {(const void*)k_factor_half, (const void*)k_factor_mid, (const void*)k_factor_temp})
    CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  double2* G = reinterpret_cast<double2*>(f.G);
  double2* H = reinterpret_cast<double2*>(f.H);
  double2* W = reinterpret_cast<double2*>(f.W);
  k_factor_temp<<<d.L + 1, kFacThreads, smem, ctx->s>>>(g, f.Tinv, status + nchains);
  CK(cudaGetLastError());
  k_factor_half<<<2 * nchains, kFacThreads, smem, ctx->s>>>(g, G, H, W, status);
  CK(cudaGetLastError());
  k_factor_mid<<<nchains, kFacThreads, smem, ctx->s>>>(g, G, H, W, status);
  CK(cudaGetLastError());
  ctx->launches += 3;
  if (ctx->p.precision == RSC_MIXED) {
    CK(cudaMalloc(&f.Gs, nent * sizeof(float4)));
    CK(cudaMalloc(&f.Hs, nent * sizeof(float4)));
    CK(cudaMalloc(&f.Ws, nent * sizeof(float4)));
    const int nb = (int)std::min<size_t>((nent + 255) / 256, 152 * 32);
    k_split_factor<<<nb, 256, 0, ctx->s>>>(G, f.Gs, (long)nent);
    k_split_factor<<<nb, 256, 0, ctx->s>>>(H, f.Hs, (long)nent);
    k_split_factor<<<nb, 256, 0, ctx->s>>>(W, f.Ws, (long)nent);
    CK(cudaGetLastError());
    ctx->launches += 3;
  }
  std::vector<int> hs(nchains + 1);
  CK(cudaMemcpyAsync(hs.data(), status, hs.size() * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  cudaFree(status);
  for (int c = 0; c <= nchains; ++c)
    if (hs[c]) {
      ctx->err = c < nchains ? "singular block in the implicit operator (chain " + std::to_string(c) + ")"
                             : std::string("singular temperature block");
      return RSC_ESINGULAR;
    }
  return RSC_OK;
}

// Factorise dt into f (FP64 factors, their double-float copies on a mixed context, the
// partitioned extras when chain_parts > 1).
rsc_status build_factor_into(rsc_ctx* ctx, double dt, DevFactor& f) {
  const auto t_fac0 = std::chrono::steady_clock::now();
  if (factor_on_device(ctx)) {
    CKS(gpu_factor(ctx, dt, f));
    ctx->factor_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_fac0).count();
    ctx->factor_on_gpu = 1;
    f.dt = dt;
    f.valid = true;
    return RSC_OK;
  }
  HostFactor hf;
  const int bad = build_factor(ctx->p, ctx->d, ctx->t, dt, hf);
  if (bad) {
    ctx->err = "singular block in the implicit operator (chain " + std::to_string(bad - 1) + ")";
    return RSC_ESINGULAR;
  }
  CKS(upload(ctx, &f.chain_off, hf.chain_off.data(), hf.chain_off.size()));
  static_assert(sizeof(cplx) == sizeof(double2), "complex layout");
  CKS(upload(ctx, &f.G, reinterpret_cast<const double2*>(hf.G.data()), hf.G.size()));
  CKS(upload(ctx, &f.H, reinterpret_cast<const double2*>(hf.H.data()), hf.H.size()));
  CKS(upload(ctx, &f.W, reinterpret_cast<const double2*>(hf.W.data()), hf.W.size()));
  CKS(upload(ctx, &f.Tinv, hf.Tinv.data(), hf.Tinv.size()));
  if (ctx->p.precision == RSC_MIXED) {
    // double-float copies for the mixed path (chain_df.cuh): hi = the entry rounded to FP32,
    // lo = the remainder rounded to FP32
    auto split_upload = [&](const std::vector<cplx>& src, float4** dst) -> rsc_status {
      std::vector<float4> t(src.size());
      for (size_t i = 0; i < src.size(); ++i) {
        const double re = src[i].real(), im = src[i].imag();
        const float rh = (float)re, ih = (float)im;
        t[i] = make_float4(rh, ih, (float)(re - (double)rh), (float)(im - (double)ih));
      }
      return upload(ctx, dst, t.data(), t.size());
    };
    if (ctx->chain_parts > 1) {
      // the double-float solve on partitioned chains: its own factorisation
      HostFactor hp;
      if (build_factor(ctx->p, ctx->d, ctx->t, dt, hp, ctx->chain_parts)) {
        ctx->err = "singular block in the partitioned implicit operator";
        return RSC_ESINGULAR;
      }
      CKS(split_upload(hp.G, &f.Gs));
      CKS(split_upload(hp.H, &f.Hs));
      CKS(split_upload(hp.W, &f.Ws));
      if (!hp.parts.empty() && !hp.unk_row.empty()) {
        f.npart = (int)(hp.parts.size() / 6);
        f.nz = (int)hp.unk_row.size();
        for (int v : hp.red_nu) f.nu_max = std::max(f.nu_max, v);
        CKS(split_upload(hp.V, &f.Vsp));
        CKS(split_upload(hp.Wsp, &f.Wsp));
        CKS(split_upload(hp.red, &f.red));
        CKS(upload(ctx, &f.parts, hp.parts.data(), hp.parts.size()));
        CKS(upload(ctx, &f.red_off, hp.red_off.data(), hp.red_off.size()));
        CKS(upload(ctx, &f.red_nu, hp.red_nu.data(), hp.red_nu.size()));
        CKS(upload(ctx, &f.zoff, hp.zoff.data(), hp.zoff.size()));
        CKS(upload(ctx, &f.unk_row, hp.unk_row.data(), hp.unk_row.size()));
        CKS(upload(ctx, &f.blk_z, hp.blk_z.data(), hp.blk_z.size()));
        CK(cudaMalloc(&f.zbuf, (size_t)f.nz * ctx->d.Nr * sizeof(double2)));
      }
    } else {
      CKS(split_upload(hf.G, &f.Gs));
      CKS(split_upload(hf.H, &f.Hs));
      CKS(split_upload(hf.W, &f.Ws));
    }
  }
  ctx->factor_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_fac0).count();
  ctx->factor_on_gpu = 0;
  f.dt = dt;
  f.valid = true;
  return RSC_OK;
}


// The double-float solve runs on odd-even reduced chains (chain_cr.cuh) on this context.
bool cr_wanted(const rsc_ctx* ctx) {
  return ctx->p.precision == RSC_MIXED && ctx->chain_cr && ctx->chain_parts == 1 &&
         !ctx->p.explicit_coriolis;
}

// Double-float copy of complex FP64 blocks: hi = the entry rounded to FP32, lo = the
// remainder rounded to FP32.
rsc_status upload_split(rsc_ctx* ctx, const std::vector<cplx>& src, float4** dst) {
  std::vector<float4> t(src.size());
  for (size_t i = 0; i < src.size(); ++i) {
    const double re = src[i].real(), im = src[i].imag();
    const float rh = (float)re, ih = (float)im;
    t[i] = make_float4(rh, ih, (float)(re - (double)rh), (float)(im - (double)ih));
  }
  return upload(ctx, dst, t.data(), t.size());
}

FacGeom fac_geom(const rsc_ctx* ctx, double dt);

// The reduced factors of f->dt on the device (cr_factor_gpu.cuh): FP64 block LU of the odd
// blocks, the reduced chains' blocks, their twisted factors, then the double-float copies.
// Needs the context's pair lists (ensure_cr).
rsc_status gpu_factor_cr(rsc_ctx* ctx, DevFactor* f) {
  const Dims& d = ctx->d;
  const int nchains = 2 * d.nm;
  std::vector<long> oo(nchains + 1), ro(nchains + 1);
  long no = 0, nr = 0;
  for (int c = 0; c < nchains; ++c) {
    const int nb = d.L - ctx->t.m_of[c / 2] + 1;
    oo[c] = no;
    ro[c] = nr;
    no += nb / 2;
    nr += (nb + 1) / 2;
  }
  oo[nchains] = no;
  ro[nchains] = nr;
  CKS(upload(ctx, &f->cr_odd_off, oo.data(), oo.size()));
  CKS(upload(ctx, &f->cr_red_off, ro.data(), ro.size()));
  const size_t blk = (size_t)d.Nr * d.Nr;
  const size_t eo = std::max<size_t>(1, no * blk), er = (size_t)nr * blk;
  double2 *Di = nullptr, *Pm = nullptr, *Qm = nullptr, *Dr = nullptr, *Ar = nullptr, *Cr = nullptr;
  double2 *G = nullptr, *H = nullptr, *W = nullptr;
  int* status = nullptr;
  double2** bufs[] = {&Di, &Pm, &Qm, &Dr, &Ar, &Cr, &G, &H, &W};
  const size_t sizes[] = {eo, eo, eo, er, er, er, er, er, er};
  auto release = [&]() {
    for (double2** b : bufs) cudaFree(*b);
    cudaFree(status);
  };
  for (int q = 0; q < 9; ++q)
    if (cudaMalloc(bufs[q], sizes[q] * sizeof(double2)) != cudaSuccess) {
      release();
      ctx->err = "cudaMalloc of the reduced-chain factorisation scratch failed";
      return RSC_ENOMEM;
    }
  cudaError_t e = cudaMalloc(&status, nchains * sizeof(int));
  auto ok = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  ok(cudaMemsetAsync(status, 0, nchains * sizeof(int), ctx->s));
  ok(cudaMemsetAsync(Qm, 0, eo * sizeof(double2), ctx->s));   // absent at a chain's last block
  ok(cudaMemsetAsync(H, 0, er * sizeof(double2), ctx->s));    // absent at the end blocks
  ok(cudaMemsetAsync(W, 0, er * sizeof(double2), ctx->s));
  const FacGeom g = fac_geom(ctx, f->dt);
  CrFacGeom cg;
  cg.pair_l = ctx->d_pair_l;
  cg.pair_m = ctx->d_pair_m;
  cg.Ms = d.Ms;
  cg.odd_off = f->cr_odd_off;
  cg.red_off = f->cr_red_off;
  const size_t smem = fac_smem_bytes(d.Nr);
  for (const void* fn : {(const void*)k_cr_fac_odd, (const void*)k_cr_fac_reduce,
                         (const void*)k_cr_fac_half, (const void*)k_cr_fac_mid})
    ok(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (e == cudaSuccess && ctx->n_cr_odd > 0) {
    cg.pairs = ctx->d_cr_pairs;
    k_cr_fac_odd<<<2 * ctx->n_cr_odd, kFacThreads, smem, ctx->s>>>(g, cg, Di, Pm, Qm, status);
    ok(cudaGetLastError());
  }
  if (e == cudaSuccess) {
    cg.pairs = ctx->d_cr_pairs + ctx->n_cr_odd;
    k_cr_fac_reduce<<<2 * ctx->n_cr_even, kFacThreads, smem, ctx->s>>>(g, cg, Pm, Qm, Dr, Ar, Cr);
    ok(cudaGetLastError());
  }
  if (e == cudaSuccess) {
    k_cr_fac_half<<<2 * nchains, kFacThreads, smem, ctx->s>>>(g, f->cr_red_off, Dr, Ar, Cr, G, H, W,
                                                            status);
    ok(cudaGetLastError());
  }
  if (e == cudaSuccess) {
    k_cr_fac_mid<<<nchains, kFacThreads, smem, ctx->s>>>(g, f->cr_red_off, Dr, Ar, Cr, G, H, W,
                                                       status);
    ok(cudaGetLastError());
  }
  // double-float copies
  float4** dsts[] = {&f->Ds, &f->Gr, &f->Hr, &f->Wr};
  const double2* srcs[] = {Di, G, H, W};
  const size_t ns[] = {eo, er, er, er};
  for (int q = 0; q < 4 && e == cudaSuccess; ++q) {
    ok(cudaMalloc(dsts[q], ns[q] * sizeof(float4)));
    if (e != cudaSuccess) break;
    const int nbk = (int)std::min<size_t>((ns[q] + 255) / 256, 152 * 32);
    k_split_factor<<<nbk, 256, 0, ctx->s>>>(srcs[q], *dsts[q], (long)ns[q]);
    ok(cudaGetLastError());
  }
  std::vector<int> hs(nchains, 0);
  if (e == cudaSuccess)
    ok(cudaMemcpyAsync(hs.data(), status, nchains * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
  ok(cudaStreamSynchronize(ctx->s));
  release();
  ctx->launches += 8;
  if (e != cudaSuccess) {
    ctx->err = std::string("CUDA error in the reduced-chain factorisation: ") + cudaGetErrorString(e);
    return RSC_ECUDA;
  }
  for (int c = 0; c < nchains; ++c)
    if (hs[c]) {
      ctx->err = "singular block in the reduced implicit operator (chain " + std::to_string(c) + ")";
      return RSC_ESINGULAR;
    }
  return RSC_OK;
}

// The reduced-chain tables of the context (pair lists, E0 / E1 as double-float pairs, the
// w buffer) on first use, and the reduced factors of f if it has none (on the GPU where the
// FP64 factorisation runs there, else on the host).
rsc_status ensure_cr(rsc_ctx* ctx, DevFactor* f) {
  const Dims& d = ctx->d;
  if (!ctx->d_E01) {
    std::vector<int> pairs;
    for (int parity = 1; parity >= 0; --parity) {
      for (int p = 0; p < d.P; ++p)
        if (((ctx->t.pair_l[p] - ctx->t.pair_m[p]) & 1) == parity) pairs.push_back(p);
      if (parity == 1) ctx->n_cr_odd = (int)pairs.size();
    }
    ctx->n_cr_even = (int)pairs.size() - ctx->n_cr_odd;
    CKS(upload(ctx, &ctx->d_cr_pairs, pairs.data(), pairs.size()));
    std::vector<float4> e((size_t)d.Nr * d.Nr);
    for (size_t i = 0; i < e.size(); ++i) {
      const double a = ctx->t.Ec[0][i], b = ctx->t.Ec[1][i];
      const float ah = (float)a, bh = (float)b;
      e[i] = make_float4(ah, (float)(a - (double)ah), bh, (float)(b - (double)bh));
    }
    CKS(upload(ctx, &ctx->d_E01, e.data(), e.size()));
    auto pair_of = [](double a, double b) {
      const float ah = (float)a, bh = (float)b;
      return make_float4(ah, (float)(a - (double)ah), bh, (float)(b - (double)bh));
    };
    std::vector<float4> rowf(d.Nr), pairf(2 * (size_t)d.P);
    for (int j = 0; j < d.Nr; ++j) {
      const double r = ctx->t.rc[j], sc = 2.0 / (r * r);
      rowf[j] = pair_of(sc / r, sc);
    }
    // normalised coefficients of the couplings to l - 1 and l + 1 (Eqs. impcor_e_final /
    // impcor_f_final, the N_l^m ratio folded in)
    for (int p = 0; p < d.P; ++p) {
      const double l = ctx->t.pair_l[p], m = ctx->t.pair_m[p], l1 = l + 1.0;
      const double a = l == 0 ? 0.0 : (l * l - 1.0) * std::sqrt((l * l - m * m) / (4.0 * l * l - 1.0));
      const double c = l == 0 ? 0.0 : l * (l + 2.0) * std::sqrt((l1 * l1 - m * m) / (4.0 * l1 * l1 - 1.0));
      pairf[2 * p] = pair_of(a * l, a);
      pairf[2 * p + 1] = pair_of(c * l1, c);
    }
    CKS(upload(ctx, &ctx->d_cr_rowf, rowf.data(), rowf.size()));
    CKS(upload(ctx, &ctx->d_cr_pairf, pairf.data(), pairf.size()));
    CK(cudaMalloc(&ctx->cr_w, (size_t)2 * 2 * d.P * d.Nr * sizeof(float4)));
  }
  if (f->Ds) return RSC_OK;
  const auto t0 = std::chrono::steady_clock::now();
  if (factor_on_device(ctx)) {
    CKS(gpu_factor_cr(ctx, f));
    f->cr_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    f->cr_on_gpu = 1;
    ctx->factor_cr_s = f->cr_s;
    ctx->factor_cr_on_gpu = 1;
    return RSC_OK;
  }
  HostFactorCR hc;
  const int bad = build_factor_cr(ctx->p, d, ctx->t, f->dt, hc);
  if (bad) {
    ctx->err = "singular block in the reduced implicit operator (chain " + std::to_string(bad - 1) + ")";
    return RSC_ESINGULAR;
  }
  CKS(upload(ctx, &f->cr_odd_off, hc.odd_off.data(), hc.odd_off.size()));
  CKS(upload(ctx, &f->cr_red_off, hc.red_off.data(), hc.red_off.size()));
  CKS(upload_split(ctx, hc.Dinv, &f->Ds));
  CKS(upload_split(ctx, hc.G, &f->Gr));
  CKS(upload_split(ctx, hc.H, &f->Hr));
  CKS(upload_split(ctx, hc.W, &f->Wr));
  f->cr_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  f->cr_on_gpu = 0;
  ctx->factor_cr_s = f->cr_s;
  ctx->factor_cr_on_gpu = 0;
  return RSC_OK;
}

rsc_status ensure_cr_locked(rsc_ctx* ctx, DevFactor* f) {
  if (!ctx->share) return ensure_cr(ctx, f);
  std::lock_guard<std::mutex> lock(ctx->share->mu);
  return ensure_cr(ctx, f);
}

rsc_status get_factor_slot(rsc_ctx* ctx, double dt, DevFactor** out);

// A shared slot gains its reduced factors under the share's lock.
rsc_status get_factor(rsc_ctx* ctx, double dt, DevFactor** out) {
  CKS(get_factor_slot(ctx, dt, out));
  return cr_wanted(ctx) ? ensure_cr_locked(ctx, *out) : RSC_OK;
}

rsc_status get_factor_slot(rsc_ctx* ctx, double dt, DevFactor** out) {
  for (auto& f : ctx->fac)
    if (f.valid && f.dt == dt) {
      *out = &f;
      return RSC_OK;
    }
  if (ctx->share && ctx->chain_parts == 1) {
    FactorShare& sh = *ctx->share;
    std::lock_guard<std::mutex> lock(sh.mu);
    for (DevFactor* f : sh.slots)
      if (f->valid && f->dt == dt) {
        *out = f;
        return RSC_OK;
      }
    if ((int)sh.slots.size() < FactorShare::kMaxSlots) {
      DevFactor* f = new (std::nothrow) DevFactor();
      if (!f) return RSC_ENOMEM;
      CK(cudaStreamSynchronize(ctx->s));
      const rsc_status st = build_factor_into(ctx, dt, *f);
      if (st != RSC_OK) {
        free_factor(*f);
        delete f;
        return st;
      }
      sh.slots.push_back(f);
      *out = f;
      return RSC_OK;
    }
  }
  DevFactor& f = ctx->fac[ctx->fac_next];
  ctx->fac_next ^= 1;
  CK(cudaStreamSynchronize(ctx->s));
  if (ctx->jvp_exec) {   // the captured Jacobian action may point into the slot being replaced
    cudaGraphExecDestroy(ctx->jvp_exec);
    ctx->jvp_exec = nullptr;
  }
  free_factor(f);
  CKS(build_factor_into(ctx, dt, f));
  *out = &f;
  return RSC_OK;
}

// ---------------------------------------------------------------------------
// Pipeline stages.
template <typename R>
rsc_status stage_synth(rsc_ctx* ctx, const double* x, void* FCout) {
  using V = typename C2<R>::T;
  const Dims& d = ctx->d;
  const DevGeom g = ctx->geom();
  {
  KSpan sp(ctx, RSC_K_RADIAL, 48.0 * d.P * d.Nr + 8.0 * d.P * d.Nd * sizeof(V),
           28.0 * d.P * d.Nd * d.Nr);
  if (sizeof(R) == 4 && ctx->radial_f32_grid > 0) {   // FP32: persistent, tables staged once
    const dim3 gr(ctx->radial_f32_grid), bl(4 * ((d.Nd + 7) / 8 * 8));
    const size_t sm = radial_f32_smem(d.Nr, d.Nd);
    const double2* xx = reinterpret_cast<const double2*>(x);
    float2* sr = reinterpret_cast<float2*>(ctx->SR);
    switch (radial_fixed(d)) {
      case 1: k_radial_f32<64, 96><<<gr, bl, sm, ctx->s>>>(g, xx, sr); break;
      case 2: k_radial_f32<96, 144><<<gr, bl, sm, ctx->s>>>(g, xx, sr); break;
      default: k_radial_f32<0, 0><<<gr, bl, sm, ctx->s>>>(g, xx, sr); break;
    }
  } else {
    k_radial<R><<<d.P, round32(std::max(d.Nd, 32)), 3 * d.Nr * sizeof(V), ctx->s>>>(
        g, reinterpret_cast<const double2*>(x), reinterpret_cast<V*>(ctx->SR));
  }
  CK(cudaGetLastError());
  }
  const LegDev<R>& L = leg<R>(ctx);
  {
  KSpan sp(ctx, RSC_K_SYNTH,
           8.0 * d.P * d.Nd * sizeof(V) + 9.0 * d.Nd * (d.K + 1) * d.nlat * sizeof(V) +
               3.0 * d.P * d.nlat2 * sizeof(R),
           52.0 * d.P * d.nlat2 * d.Nd);
  if (sizeof(R) == 4) {
    TcTables tt{ctx->tc_tiles, ctx->tc_off, ctx->tc_kpad, ctx->tc_nmt, ctx->d_status};
    const dim3 grid(d.nm, (d.Nd + kTcRadii - 1) / kTcRadii, ctx->tc_nmt);
    const bool pipe = ctx->synth_pipe != 0;
    const size_t smem = tc_synth_smem(ctx->tc_kmax, pipe);
    if (pipe)
      k_synth_tc<true><<<grid, kTcThreads, smem, ctx->s>>>(g, tt, reinterpret_cast<const float2*>(ctx->SR),
                                                    reinterpret_cast<float2*>(FCout));
    else
      k_synth_tc<false><<<grid, kTcThreads, smem, ctx->s>>>(g, tt, reinterpret_cast<const float2*>(ctx->SR),
                                                     reinterpret_cast<float2*>(FCout));
    CK(cudaGetLastError());
  } else {
    const int RT = ctx->rt_synth[0];
    k_synth<R><<<dim3(d.nm, (d.Nd + RT - 1) / RT), dim3(round32(d.nlat2), RT),
                 (size_t)RT * (d.L + 1) * 8 * sizeof(V) + 16 * 3 * (size_t)d.nlat2 * sizeof(R),
                 ctx->s>>>(g, L.view(), reinterpret_cast<const V*>(ctx->SR), reinterpret_cast<V*>(FCout));
    CK(cudaGetLastError());
  }
  }
  return RSC_OK;
}

// Shared memory of the DFT + products kernel for `wpb` warps per block.
template <typename R>
size_t products_smem(const Dims& d, bool lin, int wpb) {
  using V = typename C2<R>::T;
  const int K1 = d.K + 1, NF = lin ? 18 : 9;
  return (size_t)wpb * NF * K1 * sizeof(V) + 4 * (size_t)K1 * d.nphi * sizeof(R) +
         (size_t)wpb * 4 * (d.nphi + 1) * sizeof(R);
}

// Shared memory of the Legendre analysis for RT radii per block and TC staged latitudes.
template <typename R>
size_t analysis_smem(const Dims& d, int RT, int TC) {
  using V = typename C2<R>::T;
  return (size_t)RT * 8 * d.nlat2 * sizeof(V) + (size_t)TC * 3 * (d.L + 1) * sizeof(R);
}

// Shared memory of the right-hand-side kernel for `ppb` pairs per block.
template <typename R>
size_t rhs_smem(const Dims& d, int ppb) {
  using V = typename C2<R>::T;
  return (size_t)ppb * (10 * (size_t)d.Nr * sizeof(double2) + 6 * (size_t)d.Nr * sizeof(float2) +
                        4 * (size_t)d.Nd * sizeof(V));
}

template <typename R>
rsc_status stage_products_analysis(rsc_ctx* ctx, bool lin) {
  using V = typename C2<R>::T;
  const Dims& d = ctx->d;
  const DevGeom g = ctx->geom();
  const LegDev<R>& L = leg<R>(ctx);
  const int K1 = d.K + 1;
  const int NF = lin ? 18 : 9;
  int WPB = ctx->wpb[sizeof(R) == 4 ? 1 : 0] > 0 ? ctx->wpb[sizeof(R) == 4 ? 1 : 0] : 8;
  auto smem_for = [&](int wpb) { return products_smem<R>(d, lin, wpb); };
  while (WPB > 1 && smem_for(WPB) > 190 * 1024) WPB /= 2;
  const size_t smem = smem_for(WPB);
  const int LPW = ctx->lpw[sizeof(R) == 4 ? 1 : 0];
  dim3 grid(d.Nd, (d.nlat + WPB * LPW - 1) / (WPB * LPW));
  const double npts = (double)d.Nd * d.nlat * d.nphi;
  // Jacobian actions read the base state's grid values (k_base_grid) when they are cached
  const bool ug = lin && ctx->ug_prec == (sizeof(R) == 4 ? 2 : 1);
  const int nft = ug ? 9 : NF;   // fields transformed
  {
  KSpan sp(ctx, RSC_K_PRODUCTS,
           (double)(nft + 4) * d.Nd * K1 * d.nlat * sizeof(V) + (ug ? 9.0 * npts * sizeof(R) : 0.0),
           npts * (4.0 * nft * d.K + (lin ? 60.0 : 30.0) + 16.0 * K1));
  bool done = false;
  if constexpr (sizeof(R) == 4) {
    // Jacobian actions on the small transforms of the wave workloads
    // (the kernel's gather offsets are 32-bit: 9 Nd (K + 1) nlat coefficients per field set)
    if (lin && ug && d.nphi <= 32 && K1 <= 12 && WPB <= kPlMaxWarps &&
        9.0 * d.Nd * K1 * d.nlat < 2147483647.0) {
      const float2* fc = reinterpret_cast<const float2*>(ctx->FC);
      float2* fa = reinterpret_cast<float2*>(ctx->FA);
      const float* ugp = reinterpret_cast<const float*>(ctx->UG);
      // (nphi >= 3 K + 1, so nphi <= 32 keeps K + 1 <= 11)
      if (K1 <= 8)
        k_products_lin<8><<<grid, 32 * WPB, 0, ctx->s>>>(g, L.view(), (float)ctx->p.Ek, fc, fa, LPW, ugp);
      else
        k_products_lin<12><<<grid, 32 * WPB, 0, ctx->s>>>(g, L.view(), (float)ctx->p.Ek, fc, fa, LPW, ugp);
      done = true;
    }
  }
  if (done) {
  } else if (lin)
    k_products<R, true><<<grid, 32 * WPB, smem, ctx->s>>>(
        g, L.view(), (R)ctx->p.Ek, reinterpret_cast<const V*>(ctx->FC),
        reinterpret_cast<const V*>(ctx->FCU), reinterpret_cast<V*>(ctx->FA), LPW,
        ug ? reinterpret_cast<const R*>(ctx->UG) : nullptr);
  else
    k_products<R, false><<<grid, 32 * WPB, smem, ctx->s>>>(
        g, L.view(), (R)ctx->p.Ek, reinterpret_cast<const V*>(ctx->FC), nullptr,
        reinterpret_cast<V*>(ctx->FA), LPW, nullptr);
  CK(cudaGetLastError());
  }
  {
  KSpan sp(ctx, RSC_K_ANALYSIS,
           4.0 * d.Nd * K1 * d.nlat * sizeof(V) + 4.0 * d.P * d.Nd * sizeof(V) +
               3.0 * d.P * d.nlat2 * sizeof(R),
           24.0 * d.P * d.nlat2 * d.Nd);
  const int RTa = ctx->rt_anal[sizeof(R) == 4 ? 1 : 0];
  const int TC = ctx->atc[sizeof(R) == 4 ? 1 : 0];
  if (sizeof(R) == 4 && ctx->anal_tc) {
    TaTables ta{ctx->ta_tiles, ctx->ta_off, ctx->ta_nchunk, ctx->d_status};
    k_analysis_tc<<<dim3(d.nm, (d.Nd + kTaRadii - 1) / kTaRadii), kTaThreads, ta_smem(), ctx->s>>>(
        g, ta, reinterpret_cast<const float2*>(ctx->FA), reinterpret_cast<float2*>(ctx->AR));
  } else {
    k_analysis<R><<<dim3(d.nm, (d.Nd + RTa - 1) / RTa), dim3(round32(d.L + 1), RTa),
                    analysis_smem<R>(d, RTa, TC), ctx->s>>>(
        g, L.view(), reinterpret_cast<const V*>(ctx->FA), reinterpret_cast<V*>(ctx->AR), TC);
  }
  CK(cudaGetLastError());
  }
  return RSC_OK;
}

template <typename R>
rsc_status stage_rhs(rsc_ctx* ctx, const RhsParams& rp, const double* x, const double* U,
                     const double* u_orig, double2* out, const double* xe = nullptr) {
  using V = typename C2<R>::T;
  const Dims& d = ctx->d;
  const int tuned = ctx->ppb[sizeof(R) == 4 ? 1 : 0];
  const int PPB = tuned > 0 ? tuned : std::max(1, 256 / round32(d.Nr));
  const size_t smem = rhs_smem<R>(d, PPB);
  KSpan sp(ctx, RSC_K_RHS,
           4.0 * d.P * d.Nd * sizeof(V) + (rp.J >= 0 ? 144.0 : 96.0) * d.P * d.Nr,
           d.P * (double)d.Nr * (16.0 * d.Nd + 32.0 * d.Nr));
  if constexpr (sizeof(R) == 4) {
    // Jacobian actions of the mixed path: persistent, tables staged once (k_rhs_lin)
    if (rp.mode == 1 && !rp.explicit_coriolis && ctx->rhs_lin_grid > 0) {
      const dim3 gr(ctx->rhs_lin_grid), bl(4 * ((d.Nr + 7) / 8 * 8));
      const size_t sm = rhs_lin_smem(d.Nr, d.Nd);
      const DevGeom g = ctx->geom();
      const float2* arp = reinterpret_cast<const float2*>(ctx->AR);
      const double2* xx = reinterpret_cast<const double2*>(x);
      const double2* uu = reinterpret_cast<const double2*>(U);
      switch (radial_fixed(d)) {
        case 1: k_rhs_lin<64, 96><<<gr, bl, sm, ctx->s>>>(g, rp, arp, xx, uu, u_orig, out); break;
        case 2: k_rhs_lin<96, 144><<<gr, bl, sm, ctx->s>>>(g, rp, arp, xx, uu, u_orig, out); break;
        default: k_rhs_lin<0, 0><<<gr, bl, sm, ctx->s>>>(g, rp, arp, xx, uu, u_orig, out); break;
      }
      CK(cudaGetLastError());
      return RSC_OK;
    }
  }
  k_rhs<R><<<(d.P + PPB - 1) / PPB, dim3(round32(d.Nr), PPB), smem, ctx->s>>>(
      ctx->geom(), rp, reinterpret_cast<const V*>(ctx->AR), reinterpret_cast<const double2*>(x),
      reinterpret_cast<const double2*>(U), u_orig,
      reinterpret_cast<const double2*>(xe ? xe : x), out);
  CK(cudaGetLastError());
  return RSC_OK;
}

// MAXQ (columns per lane, 8 lanes per row) rounded up to an instantiated size.
int chain_maxq(int Nr) {
  const int q = (Nr + 7) / 8;
  return q <= 2 ? 2 : q <= 4 ? 4 : q <= 8 ? 8 : q <= 12 ? 12 : 16;
}

// Dynamic shared memory of the chain sweeps: vectors, plus this CTA's rows of every swept
// block (a sweep has at most (L + 1) / 2 + 1 steps).
size_t chain_smem(const Dims& d, int CS, bool outward) {
  const int RPC = (d.Nr + CS - 1) / CS;
  const int steps = (d.L + 2) / 2 + 1;
  return ((outward ? 4 : 2) * (size_t)d.Nr + (size_t)steps * RPC) * sizeof(double2);
}

// Dynamic shared memory of the asynchronous-exchange sweeps (chain_async.cuh).
int chain_steps_cap(const Dims& d) { return (d.L + 2) / 2 + 1; }
size_t chain_smem_async(const Dims& d, int CS, bool outward, int NS) {
  const int RPC = (d.Nr + CS - 1) / CS;
  return ((outward ? 4 : 2) * (size_t)d.Nr + (size_t)RPC * (NS - 1 + chain_steps_cap(d))) *
             sizeof(double2) + 16;
}

template <int Q, int NS>
cudaError_t launch_chain_async_q(rsc_ctx* ctx, const DevFactor* f, double* out, bool outward) {
  const Dims& d = ctx->d;
  const int CS = ctx->cluster;
  const int RPC = (d.Nr + CS - 1) / CS;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * 2 * d.nm * CS);
  cfg.blockDim = dim3(32 * NS * ((RPC + 3) / 4));
  cfg.dynamicSmemBytes = chain_smem_async(d, CS, outward, NS);
  cfg.stream = ctx->s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int cap = chain_steps_cap(d);
  if (outward)
    return cudaLaunchKernelEx(&cfg, k_chain_out_async<Q / NS, NS>, ctx->geom(),
                              (const long*)f->chain_off, (const double2*)f->H,
                              (const double2*)f->W, reinterpret_cast<double2*>(out),
                              (const double2*)ctx->mid, CS, cap, ctx->d_status);
  return cudaLaunchKernelEx(&cfg, k_chain_half_async<Q / NS, NS>, ctx->geom(),
                            (const long*)f->chain_off, (const double2*)f->H,
                            reinterpret_cast<double2*>(out), ctx->mid, CS, cap, ctx->d_status);
}

template <int Q>
cudaError_t launch_chain_q(rsc_ctx* ctx, const DevFactor* f, double* out, bool outward) {
  if (ctx->chain_async == 1) return launch_chain_async_q<Q, 2>(ctx, f, out, outward);
  if (ctx->chain_async == 2) {
    if constexpr (Q % 4 == 0) return launch_chain_async_q<Q, 4>(ctx, f, out, outward);
    return cudaErrorInvalidValue;
  }
  const Dims& d = ctx->d;
  const int CS = ctx->cluster;
  const int RPC = (d.Nr + CS - 1) / CS;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * 2 * d.nm * CS);
  cfg.blockDim = dim3(32 * ((RPC + 3) / 4));
  cfg.dynamicSmemBytes = chain_smem(d, CS, outward);
  cfg.stream = ctx->s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (outward)
    return cudaLaunchKernelEx(&cfg, k_chain_out<Q>, ctx->geom(), (const long*)f->chain_off,
                              (const double2*)f->H, (const double2*)f->W,
                              reinterpret_cast<double2*>(out), (const double2*)ctx->mid, CS);
  return cudaLaunchKernelEx(&cfg, k_chain_half<Q>, ctx->geom(), (const long*)f->chain_off,
                            (const double2*)f->H, reinterpret_cast<double2*>(out), ctx->mid, CS);
}

cudaError_t launch_chain(rsc_ctx* ctx, const DevFactor* f, double* out, bool outward) {
  switch (chain_maxq(ctx->d.Nr)) {
    case 2: return launch_chain_q<2>(ctx, f, out, outward);
    case 4: return launch_chain_q<4>(ctx, f, out, outward);
    case 8: return launch_chain_q<8>(ctx, f, out, outward);
    case 12: return launch_chain_q<12>(ctx, f, out, outward);
    default: return launch_chain_q<16>(ctx, f, out, outward);
  }
}

// Double-float sweeps (chain_df.cuh): NS = ctx->chain_df warps per row group, clusters of
// ctx->cluster_df CTAs; the shared-memory layout of the asynchronous FP64 sweeps.
// cr: the reduced chains of the odd-even reduced solve (every second block; chain_cr.cuh).
template <int Q, int NS>
cudaError_t launch_chain_df_q(rsc_ctx* ctx, const DevFactor* f, double* out, bool outward,
                              bool cr) {
  const Dims& d = ctx->d;
  const int CS = ctx->cluster_df;
  const int RPC = (d.Nr + CS - 1) / CS;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * (cr || !f->npart ? 2 * d.nm : f->npart) * CS);
  cfg.blockDim = dim3(32 * NS * ((RPC + 3) / 4));
  cfg.dynamicSmemBytes = chain_smem_async(d, CS, outward, NS);
  cfg.stream = ctx->s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int cap = chain_steps_cap(d);
  const long* off = cr ? f->cr_red_off : f->chain_off;
  const float4* H = cr ? f->Hr : f->Hs;
  const float4* W = cr ? f->Wr : f->Ws;
  const long* parts = cr ? nullptr : f->parts;
  const int bs = cr ? 2 : 1;
  if (outward)
    return cudaLaunchKernelEx(&cfg, k_chain_out_df<Q / NS, NS>, ctx->geom(), off, H, W,
                              reinterpret_cast<double2*>(out), (const double2*)ctx->mid, CS,
                              cap, ctx->d_status, parts, bs);
  return cudaLaunchKernelEx(&cfg, k_chain_half_df<Q / NS, NS>, ctx->geom(), off, H,
                            reinterpret_cast<double2*>(out), ctx->mid, CS, cap, ctx->d_status,
                            parts, bs);
}

template <int Q>
cudaError_t launch_chain_df_ns(rsc_ctx* ctx, const DevFactor* f, double* out, bool outward,
                               bool cr) {
  if (ctx->chain_df == 2) return launch_chain_df_q<Q, 2>(ctx, f, out, outward, cr);
  if constexpr (Q % 4 == 0)
    if (ctx->chain_df == 4) return launch_chain_df_q<Q, 4>(ctx, f, out, outward, cr);
  return cudaErrorInvalidValue;
}

cudaError_t launch_chain_df(rsc_ctx* ctx, const DevFactor* f, double* out, bool outward,
                            bool cr = false) {
  switch (chain_maxq(ctx->d.Nr)) {
    case 2: return launch_chain_df_ns<2>(ctx, f, out, outward, cr);
    case 4: return launch_chain_df_ns<4>(ctx, f, out, outward, cr);
    case 8: return launch_chain_df_ns<8>(ctx, f, out, outward, cr);
    case 12: return launch_chain_df_ns<12>(ctx, f, out, outward, cr);
    default: return launch_chain_df_ns<16>(ctx, f, out, outward, cr);
  }
}

// The passes of the odd-even reduced solve that run over every block (chain_cr.cuh):
// pass 0 = u and E0 u, E1 u of the odd blocks, 1 = b' and G' b' of the even blocks,
// 2 = the odd blocks from their neighbours.
template <int Q>
void launch_cr_pass_q(rsc_ctx* ctx, const DevFactor* f, double* out, int pass) {
  const Dims& d = ctx->d;
  const size_t v = (size_t)d.Nr * sizeof(float4);
  const int* odd = ctx->d_cr_pairs;
  const int* even = ctx->d_cr_pairs + ctx->n_cr_odd;
  double2* o = reinterpret_cast<double2*>(out);
  if (pass == 0)
    k_cr_odd_df<Q><<<2 * ctx->n_cr_odd, 256, 2 * v, ctx->s>>>(
        ctx->geom(), odd, f->cr_odd_off, f->Ds, ctx->d_E01, ctx->rhs, ctx->cr_w);
  else if (pass == 1)
    k_cr_even_df<Q><<<2 * ctx->n_cr_even, 256, 2 * v, ctx->s>>>(
        ctx->geom(), even, f->cr_red_off, f->Gr, ctx->d_cr_rowf, ctx->d_cr_pairf, ctx->rhs,
        ctx->cr_w, o);
  else
    k_cr_back_df<Q><<<2 * ctx->n_cr_odd, 256, 5 * v, ctx->s>>>(
        ctx->geom(), odd, f->cr_odd_off, f->Ds, ctx->d_E01, ctx->d_cr_rowf, ctx->d_cr_pairf,
        ctx->rhs, o);
}

void launch_cr_pass(rsc_ctx* ctx, const DevFactor* f, double* out, int pass) {
  switch (chain_maxq(ctx->d.Nr)) {
    case 2: launch_cr_pass_q<2>(ctx, f, out, pass); break;
    case 4: launch_cr_pass_q<4>(ctx, f, out, pass); break;
    case 8: launch_cr_pass_q<8>(ctx, f, out, pass); break;
    case 12: launch_cr_pass_q<12>(ctx, f, out, pass); break;
    default: launch_cr_pass_q<16>(ctx, f, out, pass); break;
  }
}

void launch_gemv_df(rsc_ctx* ctx, const DevFactor* f, double* out) {
  const Dims& d = ctx->d;
  const size_t sm = (size_t)d.Nr * sizeof(float4);
  double2* o = reinterpret_cast<double2*>(out);
  switch (chain_maxq(d.Nr)) {
    case 2: k_block_gemv_df<2><<<2 * d.P, 256, sm, ctx->s>>>(ctx->geom(), f->chain_off, f->Gs, ctx->rhs, o); break;
    case 4: k_block_gemv_df<4><<<2 * d.P, 256, sm, ctx->s>>>(ctx->geom(), f->chain_off, f->Gs, ctx->rhs, o); break;
    case 8: k_block_gemv_df<8><<<2 * d.P, 256, sm, ctx->s>>>(ctx->geom(), f->chain_off, f->Gs, ctx->rhs, o); break;
    case 12: k_block_gemv_df<12><<<2 * d.P, 256, sm, ctx->s>>>(ctx->geom(), f->chain_off, f->Gs, ctx->rhs, o); break;
    default: k_block_gemv_df<16><<<2 * d.P, 256, sm, ctx->s>>>(ctx->geom(), f->chain_off, f->Gs, ctx->rhs, o); break;
  }
}

// df: the double-float GEMV and sweeps (mixed path, when the context has double-float tables
// and chain_df is on); otherwise the FP64 kernels.
rsc_status stage_solve(rsc_ctx* ctx, const DevFactor* f, double* out, bool df = false,
                       bool temp = true) {
  df = df && f->Gs && f->Hs && f->Ws && ctx->chain_df != 0;
  const bool cr = df && cr_wanted(ctx) && f->Ds && ctx->d_E01;
  const Dims& d = ctx->d;
  // the temperature solve depends only on the right-hand side: it runs on a second stream
  // beside the e/f chain solve (sequentially while tracing, so that every launch is timed)
  const bool fork = !ctx->prof_on && temp;
  if (fork) {
    if (!ctx->s2) {
      CK(cudaStreamCreateWithFlags(&ctx->s2, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    }
    CK(cudaEventRecord(ctx->ev_fork, ctx->s));
    CK(cudaStreamWaitEvent(ctx->s2, ctx->ev_fork, 0));
    KSpan sp(ctx, RSC_K_TEMP, 0.0, 0.0);
    k_temp_solve<<<d.P, round32(d.Nr), (size_t)d.Nr * sizeof(double2), ctx->s2>>>(
        ctx->geom(), f->Tinv, ctx->rhs, reinterpret_cast<double2*>(out));
    CK(cudaGetLastError());
    CK(cudaEventRecord(ctx->ev_join, ctx->s2));
  }
  if (cr) {
    // odd-even reduced chains: odd blocks, reduced right-hand side, sweeps over the reduced
    // chains, odd blocks; blocks and vectors counted once per pass (the tables E0, E1 once)
    const double nr2 = (double)d.Nr * d.Nr, bo = 2.0 * ctx->n_cr_odd, be = 2.0 * ctx->n_cr_even;
    const double tab = nr2 * 16.0;
    {
      KSpan sp(ctx, RSC_K_CHAIN_RED, bo * nr2 * 16.0 + bo * d.Nr * 16.0 * 3.0 + tab,
               bo * nr2 * 8.0 + bo * nr2 * 4.0);
      launch_cr_pass(ctx, f, out, 0);
      CK(cudaGetLastError());
    }
    {
      KSpan sp(ctx, RSC_K_CHAIN_RED, be * nr2 * 16.0 + be * d.Nr * 16.0 * 6.0, be * nr2 * 8.0);
      launch_cr_pass(ctx, f, out, 1);
      CK(cudaGetLastError());
    }
    for (int outward = 0; outward < 2; ++outward) {
      KSpan sp(ctx, RSC_K_CHAIN_SEQ, be * nr2 * 16.0 + 2.0 * be * d.Nr * 16.0, be * nr2 * 8.0);
      CK(launch_chain_df(ctx, f, out, outward != 0, true));
    }
    {
      KSpan sp(ctx, RSC_K_CHAIN_RED, bo * nr2 * 16.0 + bo * d.Nr * 16.0 * 4.0 + tab,
               bo * nr2 * 8.0 + bo * nr2 * 4.0);
      launch_cr_pass(ctx, f, out, 2);
      CK(cudaGetLastError());
    }
  }
  if (!cr) {
    KSpan sp(ctx, RSC_K_CHAIN, 2.0 * d.P * d.Nr * d.Nr * 16.0 + 4.0 * d.P * d.Nr * 16.0,
             2.0 * d.P * d.Nr * d.Nr * 8.0);
    if (df)
      launch_gemv_df(ctx, f, out);
    else
      k_block_gemv<<<2 * d.P, 256, (size_t)d.Nr * sizeof(double2), ctx->s>>>(
          ctx->geom(), f->chain_off, f->G, ctx->rhs, reinterpret_cast<double2*>(out));
    CK(cudaGetLastError());
  }
  if (!cr && !ctx->p.explicit_coriolis) {
    // forward half-sweeps read H of about half the blocks each way, outward sweeps W
    KSpan sp(ctx, RSC_K_CHAIN_SEQ, 2.0 * d.P * d.Nr * d.Nr * 16.0 + 4.0 * d.P * d.Nr * 16.0,
             2.0 * d.P * d.Nr * d.Nr * 8.0);
    CK(df ? launch_chain_df(ctx, f, out, false) : launch_chain(ctx, f, out, false));
  }
  if (!cr && !ctx->p.explicit_coriolis) {
    KSpan sp(ctx, RSC_K_CHAIN_SEQ, 2.0 * d.P * d.Nr * d.Nr * 16.0 + 4.0 * d.P * d.Nr * 16.0,
             2.0 * d.P * d.Nr * d.Nr * 8.0);
    CK(df ? launch_chain_df(ctx, f, out, true) : launch_chain(ctx, f, out, true));
  }
  if (df && f->npart && !ctx->p.explicit_coriolis) {
    // partitioned chains: reduced systems, then the correction of every part
    KSpan sp(ctx, RSC_K_CHAIN, 16.0 * f->nz * f->nu_max * d.Nr * d.Nr + 4.0 * f->nz * d.Nr * 16.0 +
                                   2.0 * d.P * d.Nr * d.Nr * 16.0 + 4.0 * d.P * d.Nr * 16.0,
             8.0 * f->nz * f->nu_max * d.Nr * d.Nr + 2.0 * d.P * d.Nr * d.Nr * 8.0);
    k_spike_reduce_df<<<dim3((f->nu_max * d.Nr + 31) / 32, 2 * d.nm), 256,
                        (size_t)f->nu_max * d.Nr * sizeof(float4), ctx->s>>>(
        f->unk_row, f->zoff, f->red_nu, f->red_off, f->red, reinterpret_cast<const double2*>(out),
        f->zbuf, d.Nr);
    CK(cudaGetLastError());
    const size_t sm = 2 * (size_t)d.Nr * sizeof(float4);
    double2* o = reinterpret_cast<double2*>(out);
    switch (chain_maxq(d.Nr)) {
      case 2: k_spike_correct_df<2><<<2 * d.P, 256, sm, ctx->s>>>(ctx->geom(), f->chain_off, f->blk_z, f->Vsp, f->Wsp, f->zbuf, o); break;
      case 4: k_spike_correct_df<4><<<2 * d.P, 256, sm, ctx->s>>>(ctx->geom(), f->chain_off, f->blk_z, f->Vsp, f->Wsp, f->zbuf, o); break;
      case 8: k_spike_correct_df<8><<<2 * d.P, 256, sm, ctx->s>>>(ctx->geom(), f->chain_off, f->blk_z, f->Vsp, f->Wsp, f->zbuf, o); break;
      case 12: k_spike_correct_df<12><<<2 * d.P, 256, sm, ctx->s>>>(ctx->geom(), f->chain_off, f->blk_z, f->Vsp, f->Wsp, f->zbuf, o); break;
      default: k_spike_correct_df<16><<<2 * d.P, 256, sm, ctx->s>>>(ctx->geom(), f->chain_off, f->blk_z, f->Vsp, f->Wsp, f->zbuf, o); break;
    }
    CK(cudaGetLastError());
  }
  if (fork) {
    CK(cudaStreamWaitEvent(ctx->s, ctx->ev_join, 0));
    return RSC_OK;
  }
  if (!temp) return RSC_OK;
  KSpan sp(ctx, RSC_K_TEMP, (double)(d.L + 1) * d.Nr * d.Nr * 8.0 + 2.0 * d.P * d.Nr * 16.0,
           4.0 * d.P * d.Nr * d.Nr);
  k_temp_solve<<<d.P, round32(d.Nr), (size_t)d.Nr * sizeof(double2), ctx->s>>>(
      ctx->geom(), f->Tinv, ctx->rhs, reinterpret_cast<double2*>(out));
  CK(cudaGetLastError());
  return RSC_OK;
}

rsc_status launch_1d_grid(long n, int* blocks) {
  *blocks = (int)std::min<long>((n + 255) / 256, 152L * 8);
  return RSC_OK;
}

FacGeom fac_geom(const rsc_ctx* ctx, double dt) {
  FacGeom g;
  g.Nr = ctx->d.Nr;
  g.L = ctx->d.L;
  g.nm = ctx->d.nm;
  g.m_of = ctx->d_m_of;
  g.chain_off = nullptr;
  g.rc = ctx->d_rc;
  g.E0 = ctx->d_Ef[0];
  g.E1 = ctx->d_Ef[1];
  g.E2 = ctx->d_Ef[2];
  g.E4 = ctx->d_Ef[3];
  g.Ek = ctx->p.Ek;
  g.Pr = ctx->p.Pr;
  g.inv_dt = std::isfinite(dt) ? 1.0 / dt : 0.0;
  g.explicit_coriolis = ctx->p.explicit_coriolis ? 1 : 0;
  return g;
}

// The FP64 chain solve followed by ctx->refine steps of iterative refinement of the e/f
// chains: r = b - (M/dt + K) x with b in ctx->rhs (overwritten by r), x += solve(r).  The
// block Thomas sweeps multiply by explicit inverses of the equilibrated blocks; one step
// with an FP64 residual restores the accuracy of a pivoted LU (factor_gpu.cuh).
rsc_status stage_solve_fp64(rsc_ctx* ctx, const DevFactor* f, double* out) {
  CKS(stage_solve(ctx, f, out, false));
  const Dims& d = ctx->d;
  const long nef = 4L * d.P * d.Nr;   // doubles of the e and f fields
  int nb;
  launch_1d_grid(nef, &nb);
  for (int it = 0; it < ctx->refine; ++it) {
    {
      KSpan sp(ctx, RSC_K_CHAIN, 3.0 * d.n() * 8.0 + 4.0 * d.Nr * d.Nr * 8.0,
               2.0 * d.P * d.Nr * d.Nr * 12.0);
      k_chain_residual<<<d.P, dim3(round32(d.Nr), 2), 6 * (size_t)d.Nr * sizeof(double2), ctx->s>>>(
          fac_geom(ctx, f->dt), ctx->d_pair_l, ctx->d_pair_m, d.P,
          reinterpret_cast<const double2*>(out), ctx->rhs);
      CK(cudaGetLastError());
    }
    CKS(stage_solve(ctx, f, ctx->ref_tmp, false, false));
    {
      KSpan sp(ctx, RSC_K_BLAS, 24.0 * nef, 2.0 * nef);
      k_axpby<<<nb, 256, 0, ctx->s>>>(1.0, ctx->ref_tmp, 1.0, out, nef);
      CK(cudaGetLastError());
    }
  }
  return RSC_OK;
}

// The solve of a step or Jacobian action in transform precision R: the refined FP64 solve
// for R = double, the solve of the mixed path (double-float chains unless chain_df = 0)
// for R = float.
template <typename R>
rsc_status stage_solve_path(rsc_ctx* ctx, const DevFactor* f, double* out) {
  if (sizeof(R) == 8) return stage_solve_fp64(ctx, f, out);
  return stage_solve(ctx, f, out, true);
}

bool cluster_ok_pair(const Dims& d, int CS, int NS, const void* const (&fns)[2]);

// Whether the device can co-schedule clusters of CS CTAs for the asynchronous sweeps.
template <int Q, int NS>
bool cluster_ok_async(const Dims& d, int CS) {
  const void* const fns[2] = {(const void*)k_chain_half_async<Q / NS, NS>,
                              (const void*)k_chain_out_async<Q / NS, NS>};
  return cluster_ok_pair(d, CS, NS, fns);
}

// The same for the double-float sweeps (same shared-memory layout and block shape).
template <int Q, int NS>
bool cluster_ok_df(const Dims& d, int CS) {
  const void* const fns[2] = {(const void*)k_chain_half_df<Q / NS, NS>,
                              (const void*)k_chain_out_df<Q / NS, NS>};
  return cluster_ok_pair(d, CS, NS, fns);
}

bool cluster_ok_pair(const Dims& d, int CS, int NS, const void* const (&fns)[2]) {
  for (int w = 0; w < 2; ++w) {
    cudaFuncSetAttribute(fns[w], cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaGetLastError();
    const size_t smem = chain_smem_async(d, CS, w == 1, NS);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fns[w], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    const int RPC = (d.Nr + CS - 1) / CS;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * 2 * d.nm * CS);
    cfg.blockDim = dim3(32 * NS * ((RPC + 3) / 4));
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cfg.blockDim.x > 1024 ||
        cudaOccupancyMaxActiveClusters(&n, fns[w], &cfg) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      return false;
    }
  }
  return true;
}

bool chain_config_ok(const Dims& d, int CS, int async_mode);

// Largest cluster (16, else 8, 4, 2) that the device can co-schedule for the chain sweeps.
template <int Q>
bool cluster_ok(const Dims& d, int CS) {
  const void* fns[2] = {(const void*)k_chain_half<Q>, (const void*)k_chain_out<Q>};
  for (int w = 0; w < 2; ++w) {
    cudaFuncSetAttribute(fns[w], cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaGetLastError();
    const size_t smem = chain_smem(d, CS, w == 1);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fns[w], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    const int RPC = (d.Nr + CS - 1) / CS;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * 2 * d.nm * CS);
    cfg.blockDim = dim3(32 * ((RPC + 3) / 4));
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fns[w], &cfg) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      return false;
    }
  }
  return true;
}

rsc_status choose_cluster(rsc_ctx* ctx) {
  const Dims& d = ctx->d;
  for (int CS : {16, 8, 4, 2}) {
    if (CS > d.Nr) continue;
    bool ok = false;
    switch (chain_maxq(d.Nr)) {
      case 2: ok = cluster_ok<2>(d, CS); break;
      case 4: ok = cluster_ok<4>(d, CS); break;
      case 8: ok = cluster_ok<8>(d, CS); break;
      case 12: ok = cluster_ok<12>(d, CS); break;
      default: ok = cluster_ok<16>(d, CS); break;
    }
    if (ok) {
      ctx->cluster = CS;
      return RSC_OK;
    }
  }
  ctx->err = "no thread-block cluster configuration available for the chain solve";
  return RSC_ECUDA;
}

template <int Q>
bool chain_config_ok_q(const Dims& d, int CS, int async_mode) {
  if (async_mode == 0) return cluster_ok<Q>(d, CS);
  if (async_mode == 1) return cluster_ok_async<Q, 2>(d, CS);
  if constexpr (Q % 4 == 0) return async_mode == 2 && cluster_ok_async<Q, 4>(d, CS);
  return false;
}

template <int Q>
bool chain_df_ok_q(const Dims& d, int CS, int ns) {
  if (ns == 2) return cluster_ok_df<Q, 2>(d, CS);
  if constexpr (Q % 4 == 0) return ns == 4 && cluster_ok_df<Q, 4>(d, CS);
  return false;
}

// Double-float sweeps with ns warps per row group on clusters of CS (ns = 0: off).
bool chain_df_ok(const Dims& d, int CS, int ns) {
  if (ns == 0) return true;
  if (CS < 1 || CS > d.Nr || (ns != 2 && ns != 4)) return false;
  switch (chain_maxq(d.Nr)) {
    case 2: return chain_df_ok_q<2>(d, CS, ns);
    case 4: return chain_df_ok_q<4>(d, CS, ns);
    case 8: return chain_df_ok_q<8>(d, CS, ns);
    case 12: return chain_df_ok_q<12>(d, CS, ns);
    default: return chain_df_ok_q<16>(d, CS, ns);
  }
}

bool chain_config_ok(const Dims& d, int CS, int async_mode) {
  if (CS > d.Nr || async_mode < 0 || async_mode > 2) return false;
  switch (chain_maxq(d.Nr)) {
    case 2: return chain_config_ok_q<2>(d, CS, async_mode);
    case 4: return chain_config_ok_q<4>(d, CS, async_mode);
    case 8: return chain_config_ok_q<8>(d, CS, async_mode);
    case 12: return chain_config_ok_q<12>(d, CS, async_mode);
    default: return chain_config_ok_q<16>(d, CS, async_mode);
  }
}

RhsParams make_rp(rsc_ctx* ctx, double dt, double C, int mode) {
  RhsParams rp;
  rp.inv_dt = std::isfinite(dt) ? 1.0 / dt : 0.0;
  rp.C = C;
  rp.J = -1;
  rp.Ek = ctx->p.Ek;
  rp.Ra = ctx->p.Ra;
  rp.r_out = ctx->d.r_out;
  rp.mode = mode;
  rp.explicit_coriolis = ctx->p.explicit_coriolis ? 1 : 0;
  return rp;
}

// One IMEX step in place, transforms in precision R.
template <typename R>
rsc_status do_step(rsc_ctx* ctx, double* U, double C, double dt) {
  DevFactor* f = nullptr;
  CKS(get_factor(ctx, dt, &f));
  CKS(stage_synth<R>(ctx, U, ctx->FC));
  CKS(stage_products_analysis<R>(ctx, false));
  CKS(stage_rhs<R>(ctx, make_rp(ctx, dt, C, 0), U, nullptr, nullptr, ctx->rhs));
  CKS(stage_solve_path<R>(ctx, f, U));
  return RSC_OK;
}



// One second-order step in the laboratory frame, in place (Crank-Nicolson for the
// implicit operator, Heun's predictor-corrector for the explicit terms; the time-stepping
// scheme of Sec. 5).  Each Crank-Nicolson solve
//     (M/dt + K/2) x' = (M/dt - K/2) x + N
// is carried out as the half step (M (2/dt) + K) y = (2/dt) M x + N, x' = 2 y - x, whose
// boundary rows are (bc + B x)/2; so both solves use the factorisation at dt/2 and the
// right-hand-side kernel of the Euler step, and K x is never formed.  Predictor: N = N(x);
// corrector: N = (N(x) + N(x*))/2 with the products averaged after analysis and the
// linear explicit terms (buoyancy, explicit Coriolis) taken at (x + x*)/2.
template <typename R>
rsc_status do_step2(rsc_ctx* ctx, double* U, double dt) {
  using V = typename C2<R>::T;
  const long n = ctx->d.n();
  const long nar = (long)ctx->d.P * ctx->d.Nd * 4;
  int nb;
  launch_1d_grid(n, &nb);
  DevFactor* f = nullptr;
  CKS(get_factor(ctx, 0.5 * dt, &f));
  const RhsParams rp = make_rp(ctx, 0.5 * dt, 0.0, 3);
  // predictor: x* = 2 y* - x
  CKS(stage_synth<R>(ctx, U, ctx->FC));
  CKS(stage_products_analysis<R>(ctx, false));
  CK(cudaMemcpyAsync(ctx->AR0, ctx->AR, nar * sizeof(V), cudaMemcpyDeviceToDevice, ctx->s));
  CKS(stage_rhs<R>(ctx, rp, U, nullptr, nullptr, ctx->rhs));
  CKS(stage_solve_path<R>(ctx, f, ctx->vtmp));
  {
    KSpan sp(ctx, RSC_K_BLAS, 24.0 * n, 2.0 * n);
    k_axpby<<<nb, 256, 0, ctx->s>>>(-1.0, U, 2.0, ctx->vtmp, n);
    CK(cudaGetLastError());
  }
  // corrector
  CKS(stage_synth<R>(ctx, ctx->vtmp, ctx->FC));
  CKS(stage_products_analysis<R>(ctx, false));
  {
    KSpan sp(ctx, RSC_K_BLAS, 3.0 * nar * sizeof(V), 2.0 * nar);
    k_average<R><<<nb, 256, 0, ctx->s>>>(reinterpret_cast<V*>(ctx->AR),
                                        reinterpret_cast<const V*>(ctx->AR0), nar);
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(ctx->xtmp, U, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->s));
  {
    KSpan sp(ctx, RSC_K_BLAS, 24.0 * n, 2.0 * n);
    k_axpby<<<nb, 256, 0, ctx->s>>>(0.5, ctx->vtmp, 0.5, ctx->xtmp, n);
    CK(cudaGetLastError());
  }
  CKS(stage_rhs<R>(ctx, rp, U, nullptr, nullptr, ctx->rhs, ctx->xtmp));
  CKS(stage_solve_path<R>(ctx, f, ctx->vtmp));
  {
    KSpan sp(ctx, RSC_K_BLAS, 24.0 * n, 2.0 * n);
    k_axpby<<<nb, 256, 0, ctx->s>>>(2.0, ctx->vtmp, -1.0, U, n);
    CK(cudaGetLastError());
  }
  return RSC_OK;
}

rsc_status step_any(rsc_ctx* ctx, double* U, double C, double dt, bool fp32) {
  return fp32 ? do_step<float>(ctx, U, C, dt) : do_step<double>(ctx, U, C, dt);
}

// The base state's grid values UG from FCU (once per base state).
template <typename R>
rsc_status base_grid(rsc_ctx* ctx) {
  using V = typename C2<R>::T;
  const Dims& d = ctx->d;
  const int K1 = d.K + 1, WPB = 8;
  KSpan sp(ctx, RSC_K_PRODUCTS,
           9.0 * d.Nd * K1 * d.nlat * sizeof(V) + 9.0 * d.Nd * d.nlat * d.nphi * sizeof(R),
           (double)d.Nd * d.nlat * d.nphi * 36.0 * K1);
  k_base_grid<R><<<dim3(d.Nd, (d.nlat + WPB - 1) / WPB), 32 * WPB,
                   (size_t)WPB * 9 * K1 * sizeof(V), ctx->s>>>(
      ctx->geom(), leg<R>(ctx).view(), reinterpret_cast<const V*>(ctx->FCU),
      reinterpret_cast<R*>(ctx->UG));
  CK(cudaGetLastError());
  ctx->ug_prec = sizeof(R) == 4 ? 2 : 1;
  return RSC_OK;
}

// Base-state grid coefficients (and grid values) for Jacobian actions.
rsc_status cache_base(rsc_ctx* ctx, const double* U, bool fp32) {
  ctx->ug_prec = 0;
  if (fp32) {
    CKS(stage_synth<float>(ctx, U, ctx->FCU));
    return base_grid<float>(ctx);
  }
  CKS(stage_synth<double>(ctx, U, ctx->FCU));
  return base_grid<double>(ctx);
}

// out = (B_U - I) u with the drift unknown in slot J (Sec. 3.4); base cached.
template <typename R>
rsc_status do_jvp_eager(rsc_ctx* ctx, const double* U, double C, long J, const double* u,
                        double* out, DevFactor* f, double dt) {
  const long n = ctx->d.n();
  int nb;
  launch_1d_grid(n, &nb);
  {
    KSpan sp(ctx, RSC_K_BLAS, 16.0 * n, 0.0);
    k_copy_zero_slot<<<nb, 256, 0, ctx->s>>>(u, J, ctx->xtmp, n);
    CK(cudaGetLastError());
  }
  CKS(stage_synth<R>(ctx, ctx->xtmp, ctx->FC));
  CKS(stage_products_analysis<R>(ctx, true));
  RhsParams rp = make_rp(ctx, dt, C, 1);
  rp.J = J;  // c = u[J] is read on the device
  CKS(stage_rhs<R>(ctx, rp, ctx->xtmp, U, u, ctx->rhs));
  CKS(stage_solve_path<R>(ctx, f, out));
  {
    KSpan sp(ctx, RSC_K_BLAS, 24.0 * n, 2.0 * n);
    k_axpby<<<nb, 256, 0, ctx->s>>>(-1.0, ctx->xtmp, 1.0, out, n);
    CK(cudaGetLastError());
  }
  return RSC_OK;
}

// The same sequence with input / output through device pointer slots, for capture.
template <typename R>
rsc_status jvp_body_indirect(rsc_ctx* ctx, const double* U, double C, long J, DevFactor* f,
                             double dt) {
  const long n = ctx->d.n();
  int nb;
  launch_1d_grid(n, &nb);
  {
    KSpan sp(ctx, RSC_K_BLAS, 16.0 * n, 0.0);
    k_copy_zero_slot_ind<<<nb, 256, 0, ctx->s>>>(ctx->d_slots, J, ctx->xtmp, ctx->d_cslot, n);
    CK(cudaGetLastError());
  }
  CKS(stage_synth<R>(ctx, ctx->xtmp, ctx->FC));
  CKS(stage_products_analysis<R>(ctx, true));
  RhsParams rp = make_rp(ctx, dt, C, 1);
  rp.J = J >= 0 ? 0 : -1;  // c is read from d_cslot[0]
  CKS(stage_rhs<R>(ctx, rp, ctx->xtmp, U, ctx->d_cslot, ctx->rhs));
  CKS(stage_solve_path<R>(ctx, f, ctx->jvp_y));
  {
    KSpan sp(ctx, RSC_K_BLAS, 24.0 * n, 2.0 * n);
    k_finish_ind<<<nb, 256, 0, ctx->s>>>(ctx->d_slots, ctx->jvp_y, ctx->xtmp, n);
    CK(cudaGetLastError());
  }
  return RSC_OK;
}

template <typename R>
rsc_status do_jvp(rsc_ctx* ctx, const double* U, double C, long J, const double* u, double* out,
                  double dt) {
  DevFactor* f = nullptr;
  CKS(get_factor(ctx, dt, &f));
  if (ctx->prof_on) return do_jvp_eager<R>(ctx, U, C, J, u, out, f, dt);
  const int fp32 = sizeof(R) == 4;
  const bool same = ctx->jvp_exec && ctx->jvp_key.fp32 == fp32 && ctx->jvp_key.U == U &&
                    ctx->jvp_key.C == C && ctx->jvp_key.J == J && ctx->jvp_key.dt == dt;
  if (!same) {
    if (ctx->jvp_exec) {
      cudaGraphExecDestroy(ctx->jvp_exec);
      ctx->jvp_exec = nullptr;
    }
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    cudaStream_t user = ctx->s;
    ctx->s = ctx->cap_stream;
    const long before = ctx->launches;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(ctx->s, cudaStreamCaptureModeThreadLocal));
    const rsc_status st = jvp_body_indirect<R>(ctx, U, C, J, f, dt);
    const cudaError_t ce = cudaStreamEndCapture(ctx->s, &graph);
    ctx->s = user;
    if (st != RSC_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    CK(ce);
    const cudaError_t ie = cudaGraphInstantiate(&ctx->jvp_exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ie);
    ctx->jvp_nodes = ctx->launches - before;
    ctx->launches = before;
    ctx->jvp_key = {fp32, U, C, J, dt};
  }
  k_set_ptrs<<<1, 1, 0, ctx->s>>>(ctx->d_slots, u, out);
  CK(cudaGetLastError());
  CK(cudaGraphLaunch(ctx->jvp_exec, ctx->s));
  ctx->launches += ctx->jvp_nodes + 1;
  return RSC_OK;
}

rsc_status jvp_any(rsc_ctx* ctx, const double* U, double C, long J, const double* u, double* out,
                   double dt, bool fp32) {
  return fp32 ? do_jvp<float>(ctx, U, C, J, u, out, dt) : do_jvp<double>(ctx, U, C, J, u, out, dt);
}

// dots[j] = V_j . w for j < nv (written to ctx->dots on the device)
rsc_status dots(rsc_ctx* ctx, const double* V, long ld, int nv, const double* w, long n,
                double* dst) {
  // the split kernel needs an even length and 16-byte aligned rows (n and ld even)
  const bool split = (n % 2 == 0) && (ld % 2 == 0) &&
                     ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(w)) & 15) == 0;
  const int nchunk = split ? (int)((n + 4095) / 4096) : (int)((n + 2047) / 2048);
  {
    KSpan sp(ctx, RSC_K_DOTS, 8.0 * n * (nv + 1), 2.0 * n * nv);
    if (split)
      k_dots_split<<<dim3(nchunk, (nv + 7) / 8), 256, 0, ctx->s>>>(V, ld, nv, w, n, ctx->partial);
    else
      k_dots_tiled<<<nchunk, 256, 8 * (size_t)nv * sizeof(double), ctx->s>>>(V, ld, nv, w, n,
                                                                           ctx->partial);
    CK(cudaGetLastError());
  }
  {
    KSpan sp(ctx, RSC_K_DOTS, 8.0 * nv * nchunk, (double)nv * nchunk);
    k_reduce_rows<<<nv, 256, 0, ctx->s>>>(ctx->partial, nchunk, dst);
    CK(cudaGetLastError());
  }
  return RSC_OK;
}

// Krylov basis: kmax + 1 columns of ldV doubles, ldV = n rounded up to a multiple of 1024,
// zero-filled once so that the padding of every column stays zero.
rsc_status ensure_krylov(rsc_ctx* ctx, int kmax) {
  if (ctx->V_cols >= kmax + 1) return RSC_OK;
  CK(cudaStreamSynchronize(ctx->s));
  cudaFree(ctx->V);
  cudaFree(ctx->Vs);
  ctx->V = nullptr;
  ctx->Vs = nullptr;
  ctx->V_cols = 0;
  const long n = ctx->d.n();
  ctx->ldV = (n + 1023) / 1024 * 1024;
  const size_t bytes = (size_t)(kmax + 1) * ctx->ldV * sizeof(double);
  static_assert(sizeof(float2) == sizeof(double), "split basis layout");
  if (cudaMalloc(&ctx->V, bytes) != cudaSuccess || cudaMalloc(&ctx->Vs, bytes) != cudaSuccess) {
    cudaFree(ctx->V);
    ctx->V = nullptr;
    ctx->Vs = nullptr;
    ctx->err = "cudaMalloc of the Krylov basis failed";
    return RSC_ENOMEM;
  }
  CK(cudaMemsetAsync(ctx->V, 0, bytes, ctx->s));
  CK(cudaMemsetAsync(ctx->Vs, 0, bytes, ctx->s));
  ctx->V_cols = kmax + 1;
  return RSC_OK;
}

// Device status word written by kernels whose bounded waits gave up.
rsc_status check_status(rsc_ctx* ctx) {
  int st = 0;
  CK(cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    ctx->err = "a bounded device wait gave up (tensor-core synthesis)";
    cudaMemset(ctx->d_status, 0, sizeof(int));
    return (rsc_status)st;
  }
  return RSC_OK;
}

rsc_status norm2(rsc_ctx* ctx, const double* v, long n, double* out) {
  CKS(dots(ctx, v, n, 1, v, n, ctx->dots));
  CK(cudaMemcpyAsync(ctx->h_pinned, ctx->dots, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  *out = std::sqrt(ctx->h_pinned[0]);
  return RSC_OK;
}

// GMRES (Saad-Schultz), zero initial guess, no restart, solving (B_U - I) x = b
// (Sec. 3.3) with modified Gram-Schmidt in its one-reduction form: iteration k
//   1. w = A v_k (one Jacobian action);
//   2. one pass over the basis gives s = V^T w and t = V^T v_k; t is the new row
//      of the strictly lower part L of V^T V;
//   3. on the host, (I + L) h = s by forward substitution: h are exactly the MGS
//      coefficients h_j = v_j . (w - sum_{i<j} h_i v_i), since the MGS projector
//      prod_j (I - v_j v_j^T) equals I - V (I + L)^{-1} V^T;
//   4. one pass w <- w - V h that also sums |w|^2, then w <- w / |w| on the device.
// |w| reaches the host with the next iteration's products, so the Hessenberg
// column k (and the convergence test) completes one iteration late; a solve that
// converges at column k has run one Jacobian action more than it uses.
// Two passes over the basis per iteration (classical Gram-Schmidt with
// re-orthogonalisation takes four) and one host synchronisation.
rsc_status gmres(rsc_ctx* ctx, const double* U, double C, long J, const double* b, double* x,
                 double dt, int kmax, double tol, bool fp32, int* iters, double* relres) {
  const long n = ctx->d.n();
  CKS(ensure_krylov(ctx, kmax));
  int nb;
  launch_1d_grid(n / 2, &nb);
  double beta;
  CKS(norm2(ctx, b, n, &beta));
  if (!std::isfinite(beta)) {
    ctx->err = "non-finite right-hand side in GMRES";
    return RSC_ENAN;
  }
  CK(cudaMemsetAsync(x, 0, n * sizeof(double), ctx->s));
  *iters = 0;
  *relres = 0.0;
  if (beta == 0.0) return RSC_OK;
  double* V = ctx->V;
  float2* Vs = ctx->Vs;
  const long ld = ctx->ldV;
  // double-float orthogonalisation needs n even (element pairs) and 16-byte aligned b and x
  const bool split = ctx->krylov_split && (n % 2 == 0) &&
                     ((reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(x)) & 15) == 0;
  {
    KSpan sp(ctx, RSC_K_BLAS, 16.0 * n, 1.0 * n);
    if (split)
      k_scale_split<<<nb, 256, 0, ctx->s>>>(b, V, Vs, n, nullptr, 0, nullptr, 1.0 / beta);
    else
      k_axpby<<<nb, 256, 0, ctx->s>>>(1.0 / beta, b, 0.0, V, n);
    CK(cudaGetLastError());
  }
  // device buffer: [0] |w|^2 of the previous iteration, [1, k+2) s, [k+2, 2k+3) t
  double* dbuf = ctx->dots;
  double* d_h = ctx->dots + (2 * kMaxKrylov + 4);
  double* h_in = ctx->h_pinned;
  double* h_out = ctx->h_pinned + (2 * kMaxKrylov + 4);
  const int nchunk = (int)(ld / 1024);
  std::vector<double> H((size_t)(kmax + 1) * kmax, 0.0), cs(kmax), sn(kmax), gvec(kmax + 1, 0.0);
  std::vector<double> Lrow((size_t)kmax * (kmax + 1) / 2 + 1, 0.0);   // packed rows of L
  auto Lr = [&](int i) { return Lrow.data() + (size_t)i * (i - 1) / 2; };   // row i, i entries
  gvec[0] = beta;
  double res = beta;
  int ncols = 0;
  for (int k = 0;; ++k) {
    const bool next = k < kmax;
    double* vk = V + (long)k * ld;
    double* w = V + (long)(k + 1) * ld;
    if (next) {
      CKS(jvp_any(ctx, U, C, J, vk, w, dt, fp32));
      {
        KSpan sp(ctx, RSC_K_DOTS, 8.0 * n * (k + 3), 4.0 * n * (k + 1));
        if (split)
          k_dots_pair_s<<<dim3(nchunk, (k + 1 + 15) / 16), 512, 0, ctx->s>>>(
              Vs, ld, k + 1, w, Vs + (long)k * ld, ctx->partial);
        else
          k_dots_pair<<<dim3(nchunk, (k + 1 + 15) / 16), 256, 0, ctx->s>>>(V, ld, k + 1, w, vk,
                                                                            ctx->partial);
        CK(cudaGetLastError());
      }
      {
        KSpan sp(ctx, RSC_K_DOTS, 16.0 * (k + 1) * nchunk, 2.0 * (k + 1) * nchunk);
        k_reduce_rows<<<2 * (k + 1), 256, 0, ctx->s>>>(ctx->partial, nchunk, dbuf + 1);
        CK(cudaGetLastError());
      }
    }
    const int nread = next ? 2 * k + 3 : 1;
    CK(cudaMemcpyAsync(h_in, dbuf, nread * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    if (k >= 1) {
      // complete column k - 1 with |w_{k-1}| and its Givens rotation
      const int c = k - 1;
      const double hn = std::sqrt(std::max(0.0, h_in[0]));
      if (!std::isfinite(hn)) {
        ctx->err = "non-finite Krylov vector";
        return RSC_ENAN;
      }
      const double a = H[(size_t)c * kmax + c];
      const double rr = std::hypot(a, hn);
      cs[c] = (rr == 0.0) ? 1.0 : a / rr;
      sn[c] = (rr == 0.0) ? 0.0 : hn / rr;
      H[(size_t)c * kmax + c] = rr;
      gvec[c + 1] = -sn[c] * gvec[c];
      gvec[c] = cs[c] * gvec[c];
      res = std::fabs(gvec[c + 1]);
      ncols = k;
      if (res <= tol * beta || hn == 0.0) break;
    }
    if (!next) break;
    // new row of L, then (I + L) h = s
    const double* sv = h_in + 1;
    const double* tv = h_in + k + 2;
    double* Lk = Lr(k);
    for (int j = 0; j < k; ++j) Lk[j] = tv[j];
    // (the GPU waits for this solve: each row's sum runs in four independent chains)
    for (int i = 0; i <= k; ++i) {
      const double* Li = Lr(i);
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int j = 0;
      for (; j + 4 <= i; j += 4) {
        a0 += Li[j] * h_out[j];
        a1 += Li[j + 1] * h_out[j + 1];
        a2 += Li[j + 2] * h_out[j + 2];
        a3 += Li[j + 3] * h_out[j + 3];
      }
      for (; j < i; ++j) a0 += Li[j] * h_out[j];
      h_out[i] = sv[i] - ((a0 + a1) + (a2 + a3));
    }
    if (!std::isfinite(h_out[k])) {
      ctx->err = "non-finite Krylov vector";
      return RSC_ENAN;
    }
    // Hessenberg column k with the earlier rotations applied (rows 0..k)
    for (int i = 0; i <= k; ++i) H[(size_t)i * kmax + k] = h_out[i];
    for (int i = 0; i < k; ++i) {
      const double a = H[(size_t)i * kmax + k], bb = H[(size_t)(i + 1) * kmax + k];
      H[(size_t)i * kmax + k] = cs[i] * a + sn[i] * bb;
      H[(size_t)(i + 1) * kmax + k] = -sn[i] * a + cs[i] * bb;
    }
    CK(cudaMemcpyAsync(d_h, h_out, (k + 1) * sizeof(double), cudaMemcpyHostToDevice, ctx->s));
    {
      KSpan sp(ctx, RSC_K_AXPY, 8.0 * n * (k + 3), 2.0 * n * (k + 2));
      if (split)
        k_axpy_norm_s<<<nb, 256, (size_t)(k + 1) * sizeof(float2), ctx->s>>>(Vs, ld, k + 1, d_h,
                                                                             w, n, ctx->partial);
      else
        k_axpy_norm<<<nb, 256, 0, ctx->s>>>(V, ld, k + 1, d_h, w, n, ctx->partial);
      CK(cudaGetLastError());
    }
    if (!split) {
      KSpan sp(ctx, RSC_K_BLAS, 8.0 * nb, 1.0 * nb);
      k_reduce_rows<<<1, 256, 0, ctx->s>>>(ctx->partial, nb, dbuf);
      CK(cudaGetLastError());
    }
    {
      KSpan sp(ctx, RSC_K_BLAS, 16.0 * n + 8.0 * nb, 1.0 * n);
      if (split)   // the norm's block shares are summed inside (|w|^2 to dbuf[0])
        k_scale_split<<<nb, 256, 0, ctx->s>>>(w, w, Vs + (long)(k + 1) * ld, n, ctx->partial, nb,
                                              dbuf, 1.0);
      else
        k_scale_inv_sqrt<<<nb, 256, 0, ctx->s>>>(w, n, dbuf);
      CK(cudaGetLastError());
    }
  }
  const int kk = ncols;
  std::vector<double> y(kk, 0.0);
  for (int i = kk - 1; i >= 0; --i) {
    double s = gvec[i];
    for (int q = i + 1; q < kk; ++q) s -= H[(size_t)i * kmax + q] * y[q];
    y[i] = s / H[(size_t)i * kmax + i];
  }
  for (int i = 0; i < kk; ++i) h_out[i] = y[i];
  CK(cudaMemcpyAsync(d_h, h_out, kk * sizeof(double), cudaMemcpyHostToDevice, ctx->s));
  {
    KSpan sp(ctx, RSC_K_AXPY, 8.0 * n * (kk + 2), 2.0 * n * kk);
    if (split)
      k_multi_axpy_s<<<nb, 256, (size_t)std::max(kk, 1) * sizeof(float2), ctx->s>>>(Vs, ld, kk,
                                                                                    d_h, x, n);
    else
      k_multi_axpy2<<<nb, 256, 0, ctx->s>>>(V, ld, kk, d_h, 1.0, x, n);
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(ctx->s));
  *iters = kk;
  *relres = res / beta;
  return RSC_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: the launch shapes of the transform, right-hand-side and chain kernels are
// picked by timing each candidate (CUDA events, 3 launches after a warm-up) on this
// context's own workspace, with the conductive state as input.
int radii_limit(const void* fn, int threads_x) {
  cudaFuncAttributes at{};
  if (cudaFuncGetAttributes(&at, fn) != cudaSuccess) return 1;
  int rt = 4;
  while (rt > 1 && ((long)rt * threads_x * std::max(at.numRegs, 1) > 65536 || rt * threads_x > 1024))
    --rt;
  return rt;
}

bool tuning_ok(rsc_ctx* ctx, const rsc_tuning& t) {
  const Dims& d = ctx->d;
  auto pow2 = [](int v, int hi) { return v >= 1 && v <= hi && (v & (v - 1)) == 0; };
  for (int p = 0; p < 2; ++p) {
    if (!pow2(t.products_warps[p], 8)) return false;
    const size_t sm = p ? products_smem<float>(d, true, t.products_warps[p])
                        : products_smem<double>(d, true, t.products_warps[p]);
    if (sm > 190 * 1024) return false;
    const int ra = radii_limit(p ? (const void*)k_analysis<float> : (const void*)k_analysis<double>,
                               round32(d.L + 1));
    if (t.analysis_radii[p] < 1 || t.analysis_radii[p] > ra) return false;
    if (t.analysis_chunk[p] < 1) return false;
    if (!pow2(t.products_lats[p], 16)) return false;
    if ((p ? analysis_smem<float>(d, t.analysis_radii[p], t.analysis_chunk[p])
           : analysis_smem<double>(d, t.analysis_radii[p], t.analysis_chunk[p])) > 200 * 1024)
      return false;
    if (!pow2(t.rhs_pairs[p], 8) ||
        !threads_fit(p ? (const void*)k_rhs<float> : (const void*)k_rhs<double>,
                     round32(d.Nr) * t.rhs_pairs[p]))
      return false;
    if ((p ? rhs_smem<float>(d, t.rhs_pairs[p]) : rhs_smem<double>(d, t.rhs_pairs[p])) > 200 * 1024)
      return false;
  }
  if (t.synth_radii < 1 || t.synth_radii > radii_limit((const void*)k_synth<double>, round32(d.nlat2)))
    return false;
  if (t.analysis_tc != 0 && t.analysis_tc != 1) return false;
  if (t.krylov_split != 0 && t.krylov_split != 1) return false;
  if (t.chain_parts < 1 || t.chain_parts > kMaxChainParts) return false;
  if (t.factor_gpu != 0 && t.factor_gpu != 1) return false;
  if (t.refine < 0 || t.refine > 2) return false;
  if (t.synth_pipe != 0 && t.synth_pipe != 1) return false;
  if (t.chain_cr != 0 && t.chain_cr != 1) return false;
  if (t.synth_pipe == 1 && !synth_pipe_fits(ctx->tc_kmax)) return false;
  if (!chain_df_ok(d, t.chain_df_cluster, t.chain_df)) return false;
  return chain_config_ok(d, t.chain_cluster, t.chain_async);
}

void get_tuning(const rsc_ctx* ctx, rsc_tuning* t) {
  const Dims& d = ctx->d;
  for (int p = 0; p < 2; ++p) {
    int w = ctx->wpb[p] > 0 ? ctx->wpb[p] : 8;
    while (w > 1 && (p ? products_smem<float>(d, true, w) : products_smem<double>(d, true, w)) >
                        190 * 1024)
      w /= 2;
    t->products_warps[p] = w;
    t->analysis_radii[p] = ctx->rt_anal[p];
    t->rhs_pairs[p] = ctx->ppb[p] > 0 ? ctx->ppb[p] : std::max(1, 256 / round32(d.Nr));
    t->analysis_chunk[p] = ctx->atc[p];
    t->products_lats[p] = ctx->lpw[p];
  }
  t->synth_radii = ctx->rt_synth[0];
  t->chain_cluster = ctx->cluster;
  t->chain_async = ctx->chain_async;
  t->analysis_tc = ctx->anal_tc;
  t->chain_df = ctx->chain_df;
  t->chain_df_cluster = ctx->cluster_df;
  t->krylov_split = ctx->krylov_split;
  t->chain_parts = ctx->chain_parts;
  t->factor_gpu = ctx->factor_gpu;
  t->refine = ctx->refine;
  t->synth_pipe = ctx->synth_pipe;
  t->chain_cr = ctx->chain_cr;
  for (int q = 0; q < 6; ++q) t->ms[q] = ctx->tune_ms[q];
}

void set_tuning(rsc_ctx* ctx, const rsc_tuning& t) {
  for (int p = 0; p < 2; ++p) {
    ctx->wpb[p] = t.products_warps[p];
    ctx->rt_anal[p] = t.analysis_radii[p];
    ctx->ppb[p] = t.rhs_pairs[p];
    ctx->atc[p] = t.analysis_chunk[p];
    ctx->lpw[p] = t.products_lats[p];
  }
  ctx->rt_synth[0] = t.synth_radii;
  ctx->cluster = t.chain_cluster;
  ctx->chain_async = t.chain_async;
  ctx->anal_tc = t.analysis_tc;
  ctx->chain_df = t.chain_df;
  ctx->cluster_df = t.chain_df_cluster;
  ctx->krylov_split = t.krylov_split;
  ctx->refine = t.refine;
  ctx->synth_pipe = t.synth_pipe;
  ctx->chain_cr = t.chain_cr;   // the reduced factors are added to a slot on its next use
  if (t.factor_gpu != ctx->factor_gpu) {
    // the factorisations are rebuilt where the new setting says
    ctx->factor_gpu = t.factor_gpu;
    cudaStreamSynchronize(ctx->s);
    for (auto& f : ctx->fac) free_factor(f);
  }
  if (t.chain_parts != ctx->chain_parts) {
    // another partition of the double-float solve: both factorisation slots are rebuilt
    ctx->chain_parts = t.chain_parts;
    cudaStreamSynchronize(ctx->s);
    for (auto& f : ctx->fac) free_factor(f);
  }
  if (ctx->jvp_exec) {   // the captured Jacobian action embeds the old launch shapes
    cudaGraphExecDestroy(ctx->jvp_exec);
    ctx->jvp_exec = nullptr;
  }
}

template <typename R>
rsc_status tune_precision(rsc_ctx* ctx, rsc_tuning& t, cudaEvent_t e0, cudaEvent_t e1) {
  const int p = sizeof(R) == 4 ? 1 : 0;
  const Dims& d = ctx->d;
  rsc_status st = RSC_OK;
  auto timeit = [&](auto&& launch) -> double {
    st = launch();
    if (st != RSC_OK) return 1e30;
    cudaEventRecord(e0, ctx->s);
    for (int r = 0; r < 3 && st == RSC_OK; ++r) st = launch();
    cudaEventRecord(e1, ctx->s);
    if (cudaEventSynchronize(e1) != cudaSuccess) st = RSC_ECUDA;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    return st == RSC_OK ? ms / 3.0 : 1e30;
  };
  CKS(stage_synth<R>(ctx, ctx->rtmp, ctx->FC));
  ctx->ug_prec = 0;
  CKS(stage_synth<R>(ctx, ctx->rtmp, ctx->FCU));
  CKS(base_grid<R>(ctx));
  auto pa = [&] { return stage_products_analysis<R>(ctx, true); };
  // products: warps per block x latitudes per warp
  double best = 1e30;
  int bw = t.products_warps[p], bl = t.products_lats[p];
  for (int w : {1, 2, 4, 8}) {
    if (products_smem<R>(d, true, w) > 190 * 1024) continue;
    for (int lp : {1, 2, 4, 8}) {
      ctx->wpb[p] = w;
      ctx->lpw[p] = lp;
      const double ms = timeit(pa);
      CKS(st);
      if (ms < best) { best = ms; bw = w; bl = lp; }
    }
  }
  ctx->wpb[p] = t.products_warps[p] = bw;
  ctx->lpw[p] = t.products_lats[p] = bl;
  // analysis: radii per block x latitudes per staged table chunk
  best = 1e30;
  int br = t.analysis_radii[p], bc = t.analysis_chunk[p];
  const int rmax = radii_limit((const void*)k_analysis<R>, round32(d.L + 1));
  for (int r = 1; r <= rmax; r *= 2) {
    for (int tc : {16, 32, 48, d.nlat2}) {
      if (tc > d.nlat2 || analysis_smem<R>(d, r, tc) > 200 * 1024) continue;
      ctx->rt_anal[p] = r;
      ctx->atc[p] = tc;
      const double ms = timeit(pa);
      CKS(st);
      if (ms < best) { best = ms; br = r; bc = tc; }
    }
  }
  ctx->rt_anal[p] = t.analysis_radii[p] = br;
  ctx->atc[p] = t.analysis_chunk[p] = bc;
  if (p == 1) {   // tensor-core analysis against the best CUDA-core shape
    ctx->anal_tc = 1;
    const double ms = timeit(pa);
    CKS(st);
    CKS(check_status(ctx));
    ctx->anal_tc = t.analysis_tc = (ms < best) ? 1 : 0;
    if (ms < best) best = ms;
  }
  if (p == 1) ctx->tune_ms[0] = best;   // products + analysis of the mixed path
  // tensor-core synthesis (mixed path): two-stage schedule against one phase at a time
  if (p == 1 && synth_pipe_fits(ctx->tc_kmax)) {
    double bt = 1e30;
    int bpipe = 0;
    for (int pipe : {0, 1}) {
      ctx->synth_pipe = pipe;
      const double ms = timeit([&] { return stage_synth<float>(ctx, ctx->rtmp, ctx->FC); });
      CKS(st);
      CKS(check_status(ctx));
      if (ms < bt) { bt = ms; bpipe = pipe; }
    }
    ctx->synth_pipe = t.synth_pipe = bpipe;
  }
  // synthesis (CUDA-core FP64 path): radii per block
  if (p == 0) {
    best = 1e30;
    int bs = t.synth_radii;
    const int smax = radii_limit((const void*)k_synth<double>, round32(d.nlat2));
    for (int r = 1; r <= smax; r *= 2) {
      ctx->rt_synth[0] = r;
      const double ms = timeit([&] { return stage_synth<double>(ctx, ctx->rtmp, ctx->FC); });
      CKS(st);
      if (ms < best) { best = ms; bs = r; }
    }
    ctx->rt_synth[0] = t.synth_radii = bs;
    ctx->tune_ms[1] = best;
  }
  // right-hand side: pairs per block (Jacobian-action mode)
  RhsParams rp = make_rp(ctx, 200.0, 0.0, 1);
  best = 1e30;
  int bp = t.rhs_pairs[p];
  for (int q : {1, 2, 4, 8}) {
    if (!threads_fit((const void*)k_rhs<R>, round32(d.Nr) * q) || rhs_smem<R>(d, q) > 200 * 1024)
      continue;
    ctx->ppb[p] = q;
    const double ms = timeit([&] { return stage_rhs<R>(ctx, rp, ctx->rtmp, ctx->rtmp, nullptr, ctx->rhs); });
    CKS(st);
    if (ms < best) { best = ms; bp = q; }
  }
  ctx->ppb[p] = t.rhs_pairs[p] = bp;
  if (p == 1) ctx->tune_ms[2] = best;
  return RSC_OK;
}

rsc_status autotune(rsc_ctx* ctx, rsc_tuning* out) {
  rsc_tuning t{};
  get_tuning(ctx, &t);
  CKS(rsc_conductive_state(ctx, ctx->rtmp));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const bool prof = ctx->prof_on;
  ctx->prof_on = false;
  rsc_status st = tune_precision<double>(ctx, t, e0, e1);
  if (st == RSC_OK) st = tune_precision<float>(ctx, t, e0, e1);
  // chain sweeps: CTAs per cluster, on the Newton factorisation (dt = 200)
  if (st == RSC_OK) {
    DevFactor* f = nullptr;
    st = get_factor(ctx, 200.0, &f);
    double best = 1e30;
    int bc = t.chain_cluster, ba = t.chain_async;
    for (int am : {0, 1, 2}) {
      for (int cs : {16, 8, 4, 2}) {
        if (st != RSC_OK) break;
        if (!chain_config_ok(ctx->d, cs, am)) continue;
        ctx->cluster = cs;
        ctx->chain_async = am;
        st = stage_solve(ctx, f, ctx->xtmp);
        cudaEventRecord(e0, ctx->s);
        for (int r = 0; r < 3 && st == RSC_OK; ++r) st = stage_solve(ctx, f, ctx->xtmp);
        cudaEventRecord(e1, ctx->s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = RSC_ECUDA;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (st == RSC_OK && ms / 3.0 < best) { best = ms / 3.0; bc = cs; ba = am; }
      }
    }
    if (st == RSC_OK) st = check_status(ctx);   // a timed-out wait of a sweep candidate
    t.chain_cluster = bc;
    t.chain_async = ba;
    ctx->cluster = bc;
    ctx->chain_async = ba;
    ctx->tune_ms[3] = best;
    // mixed path: the double-float chain solve against the best FP64 one
    if (st == RSC_OK && f->Gs) {
      double best_df = 1e30;
      int bn = 0, bcs = t.chain_df_cluster, bcr = 0;
      const int saved_cr = ctx->chain_cr;
      for (int cr : {0, 1}) {   // the unreduced chains, then the odd-even reduced ones
        ctx->chain_cr = cr;
        if (cr && (st != RSC_OK || !cr_wanted(ctx))) break;
        if (cr) st = ensure_cr_locked(ctx, f);
        for (int ns : {2, 4}) {
          for (int cs : {16, 8, 4, 2}) {
            if (st != RSC_OK) break;
            if (!chain_df_ok(ctx->d, cs, ns)) continue;
            ctx->chain_df = ns;
            ctx->cluster_df = cs;
            st = stage_solve(ctx, f, ctx->xtmp, true);
            cudaEventRecord(e0, ctx->s);
            for (int r = 0; r < 3 && st == RSC_OK; ++r) st = stage_solve(ctx, f, ctx->xtmp, true);
            cudaEventRecord(e1, ctx->s);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = RSC_ECUDA;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (st == RSC_OK && ms / 3.0 < best_df) {
              best_df = ms / 3.0;
              bn = ns;
              bcs = cs;
              bcr = cr;
            }
          }
        }
      }
      ctx->chain_cr = saved_cr;
      if (st == RSC_OK) st = check_status(ctx);
      t.chain_df = best_df < best ? bn : 0;
      t.chain_df_cluster = bcs;
      t.chain_cr = best_df < best ? bcr : 0;
      ctx->tune_ms[5] = best_df < 1e30 ? best_df : 0.0;
    }
  }
  ctx->prof_on = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != RSC_OK) return st;
  set_tuning(ctx, t);
  get_tuning(ctx, &t);
  if (out) *out = t;
  return RSC_OK;
}

// Kinetic energy and Nusselt numbers of U (diagnostics of Secs. 4-5).
rsc_status diagnostics(rsc_ctx* ctx, const double* U, double out[3]) {
  const Dims& d = ctx->d;
  if (!ctx->d_diag) {
    const int nq = 2 * d.Nr + 16;
    std::vector<double> x, w;
    gauss_legendre(nq, x, w);
    const double h = 0.5 * (d.r_out - d.r_in), dxdr = 1.0 / h;
    std::vector<double> T((size_t)nq * d.Nr), dT((size_t)nq * d.Nr), r(nq), wq(nq);
    for (int q = 0; q < nq; ++q) {
      const double th = std::acos(x[q]), st = std::sin(th);
      r[q] = h * x[q] + 0.5 * (d.r_out + d.r_in);
      wq[q] = h * w[q];
      for (int k = 0; k < d.Nr; ++k) {
        T[(size_t)q * d.Nr + k] = std::cos(k * th);
        dT[(size_t)q * d.Nr + k] = k * std::sin(k * th) / st * dxdr;   // T_k' = k U_{k-1}
      }
    }
    rsc_status st;
    if ((st = upload(ctx, &ctx->d_keT, T.data(), T.size())) != RSC_OK) return st;
    if ((st = upload(ctx, &ctx->d_kedT, dT.data(), dT.size())) != RSC_OK) return st;
    if ((st = upload(ctx, &ctx->d_ker, r.data(), r.size())) != RSC_OK) return st;
    if ((st = upload(ctx, &ctx->d_kew, wq.data(), wq.size())) != RSC_OK) return st;
    CK(cudaMalloc((void**)&ctx->d_diag, 3 * sizeof(double)));
    ctx->ke_nq = nq;
  }
  const double V = 4.0 * M_PI * (std::pow(d.r_out, 3) - std::pow(d.r_in, 3)) / 3.0;
  const double g_in = -d.r_out * d.r_in / (d.r_in * d.r_in);
  const double g_out = -d.r_out * d.r_in / (d.r_out * d.r_out);
  {
    KSpan sp(ctx, RSC_K_BLAS, 16.0 * d.P * d.Nr * 2, 12.0 * d.P * d.Nr * ctx->ke_nq);
    k_ke_pairs<<<d.P, 128, 2 * d.Nr * sizeof(double2), ctx->s>>>(
        U, d.P, d.Nr, ctx->ke_nq, ctx->d_keT, ctx->d_kedT, ctx->d_ker, ctx->d_kew, ctx->d_pair_l,
        ctx->d_pair_m, ctx->partial);
    CK(cudaGetLastError());
  }
  {
    KSpan sp(ctx, RSC_K_BLAS, 8.0 * d.P, 1.0 * d.P);
    k_diag_finish<<<1, 256, 0, ctx->s>>>(ctx->partial, d.P, U, d.Nr, 0.5 / V,
                                         2.0 / (d.r_out - d.r_in), g_in, g_out, ctx->d_diag);
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(ctx->h_pinned, ctx->d_diag, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                     ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  for (int i = 0; i < 3; ++i) out[i] = ctx->h_pinned[i];
  return RSC_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

int rsc_abi_version(void) { return RSC_ABI_VERSION; }

const char* rsc_status_string(int s) {
  switch (s) {
    case RSC_OK: return "RSC_OK";
    case RSC_EINVAL: return "RSC_EINVAL";
    case RSC_ENOMEM: return "RSC_ENOMEM";
    case RSC_ECUDA: return "RSC_ECUDA";
    case RSC_ENOCONV: return "RSC_ENOCONV";
    case RSC_ENAN: return "RSC_ENAN";
    case RSC_ESINGULAR: return "RSC_ESINGULAR";
    case RSC_ETIMEOUT: return "RSC_ETIMEOUT";
    case RSC_ERESOLUTION: return "RSC_ERESOLUTION";
    default: return "unknown status";
  }
}

const char* rsc_last_error(const rsc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

rsc_status rsc_create(const rsc_params* params, void* stream, rsc_ctx** out) {
  if (!out) return RSC_EINVAL;
  *out = nullptr;
  CKS(check_params(params));
  rsc_ctx* ctx = new (std::nothrow) rsc_ctx();
  if (!ctx) return RSC_ENOMEM;
  ctx->p = *params;
  ctx->s = reinterpret_cast<cudaStream_t>(stream);
  build_dims(ctx->p, ctx->d);
  build_tables(ctx->p, ctx->d, ctx->t);
  rsc_status st = RSC_OK;
  auto fail = [&](rsc_status s) {
    *out = ctx;  // keep the context so that rsc_last_error works; caller destroys
    return s;
  };
  const Dims& d = ctx->d;
  const HostTables& t = ctx->t;
  if (cudaGetDevice(&ctx->device) != cudaSuccess) {
    ctx->err = "no CUDA device";
    return fail(RSC_ECUDA);
  }
#define UP(dst, vec) \
  if ((st = upload(ctx, &dst, vec.data(), vec.size())) != RSC_OK) return fail(st)
  UP(ctx->d_m_of, t.m_of);
  UP(ctx->d_pstart, t.pstart);
  UP(ctx->d_pair_l, t.pair_l);
  UP(ctx->d_pair_m, t.pair_m);
  UP(ctx->d_leg_off, t.leg_off);
  UP(ctx->d_rc, t.rc);
  UP(ctx->d_rd, t.rd);
  {
    auto e0 = transpose(t.Ec[0], d.Nr, d.Nr), e2 = transpose(t.Ec[2], d.Nr, d.Nr);
    auto e1 = transpose(t.Ec[1], d.Nr, d.Nr);
    UP(ctx->d_EcT1, e1);
    UP(ctx->d_Ef[0], t.Ec[0]);
    UP(ctx->d_Ef[1], t.Ec[1]);
    UP(ctx->d_Ef[2], t.Ec[2]);
    UP(ctx->d_Ef[3], t.Ec[4]);
    auto d0 = transpose(t.Ed[0], d.Nd, d.Nr), d1 = transpose(t.Ed[1], d.Nd, d.Nr),
         d2 = transpose(t.Ed[2], d.Nd, d.Nr);
    auto r0 = transpose(t.R0, d.Nr, d.Nd), r1 = transpose(t.R1, d.Nr, d.Nd);
    UP(ctx->d_EcT0, e0);
    UP(ctx->d_EcT2, e2);
    UP(ctx->d_EdT0, d0);
    UP(ctx->d_EdT1, d1);
    UP(ctx->d_EdT2, d2);
    UP(ctx->d_R0T, r0);
    UP(ctx->d_R1T, r1);
    auto tof = [](const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); };
    auto d0f = tof(d0), d1f = tof(d1), d2f = tof(d2), r0f = tof(r0), r1f = tof(r1), rdf = tof(t.rd);
    UP(ctx->f_EdT0, d0f);
    UP(ctx->f_EdT1, d1f);
    UP(ctx->f_EdT2, d2f);
    UP(ctx->f_R0T, r0f);
    UP(ctx->f_R1T, r1f);
    UP(ctx->f_rd, rdf);
    auto e0f = tof(e0), e2f = tof(e2);
    UP(ctx->f_EcT0, e0f);
    UP(ctx->f_EcT2, e2f);
  }
#undef UP
  if ((st = upload_legendre(ctx, ctx->leg64)) != RSC_OK) return fail(st);
  if ((st = upload_legendre(ctx, ctx->leg32)) != RSC_OK) return fail(st);
  if ((st = set_smem_limits(ctx)) != RSC_OK) return fail(st);
  if ((st = build_tc_tables(ctx)) != RSC_OK) return fail(st);
  if ((st = build_ta_tables(ctx)) != RSC_OK) return fail(st);
  if (cudaMalloc((void**)&ctx->d_status, sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess) {
    ctx->err = "cudaMalloc of the status word failed";
    return fail(RSC_ENOMEM);
  }
  if ((st = choose_cluster(ctx)) != RSC_OK) return fail(st);
  if (ctx->p.precision == RSC_MIXED) {
    // double-float chain solve for the mixed path by default (rsc_autotune may keep FP64)
    for (int cs : {ctx->cluster, 8, 4, 16, 2})
      if (chain_df_ok(ctx->d, cs, 2)) {
        ctx->chain_df = 2;
        ctx->cluster_df = cs;
        break;
      }
    ctx->chain_cr = 1;   // on odd-even reduced chains (used with implicit Coriolis only)
  }
  const size_t c16 = sizeof(double2);
  const size_t K1 = d.K + 1;
  auto alloc = [&](void** p, size_t bytes) -> rsc_status {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      ctx->err = "cudaMalloc of workspace failed";
      return RSC_ENOMEM;
    }
    return RSC_OK;
  };
  const long n = d.n();
  if ((st = alloc(&ctx->SR, (size_t)d.P * d.Nd * 8 * c16)) != RSC_OK) return fail(st);
  if ((st = alloc(&ctx->FC, 9 * (size_t)d.Nd * K1 * d.nlat * c16)) != RSC_OK) return fail(st);
  if ((st = alloc(&ctx->FCU, 9 * (size_t)d.Nd * K1 * d.nlat * c16)) != RSC_OK) return fail(st);
  if ((st = alloc(&ctx->UG, 9 * (size_t)d.Nd * d.nlat * d.nphi * sizeof(double))) != RSC_OK)
    return fail(st);
  if ((st = alloc(&ctx->FA, 4 * (size_t)d.Nd * K1 * d.nlat * c16)) != RSC_OK) return fail(st);
  if ((st = alloc(&ctx->AR, (size_t)d.P * d.Nd * 4 * c16)) != RSC_OK) return fail(st);
  if ((st = alloc(&ctx->AR0, (size_t)d.P * d.Nd * 4 * c16)) != RSC_OK) return fail(st);
  if ((st = alloc((void**)&ctx->rhs, (size_t)n * sizeof(double))) != RSC_OK) return fail(st);
  if ((st = alloc((void**)&ctx->mid, (size_t)2 * d.nm * kMaxChainParts * 3 * d.Nr * c16)) != RSC_OK)
    return fail(st);
  if ((st = alloc((void**)&ctx->d_slots, 2 * sizeof(double*))) != RSC_OK) return fail(st);
  if ((st = alloc((void**)&ctx->d_cslot, sizeof(double))) != RSC_OK) return fail(st);
  if ((st = alloc((void**)&ctx->jvp_y, (size_t)n * sizeof(double))) != RSC_OK) return fail(st);
  if ((st = alloc((void**)&ctx->xtmp, (size_t)n * sizeof(double))) != RSC_OK) return fail(st);
  if ((st = alloc((void**)&ctx->vtmp, (size_t)n * sizeof(double))) != RSC_OK) return fail(st);
  if ((st = alloc((void**)&ctx->rtmp, (size_t)n * sizeof(double))) != RSC_OK) return fail(st);
  if ((st = alloc((void**)&ctx->ustate, (size_t)n * sizeof(double))) != RSC_OK) return fail(st);
  if ((st = alloc((void**)&ctx->ref_tmp, (size_t)n * sizeof(double))) != RSC_OK) return fail(st);
  ctx->nblk_dot = (int)std::max<long>((n + 1023) / 1024, 152L * 8);   // pass-A chunks, pass-B blocks
  if ((st = alloc((void**)&ctx->partial, (size_t)ctx->nblk_dot * (2 * kMaxKrylov + 4) * sizeof(double))) != RSC_OK)
    return fail(st);
  if ((st = alloc((void**)&ctx->dots, (size_t)(3 * kMaxKrylov + 8) * sizeof(double))) != RSC_OK)
    return fail(st);
  if (cudaMallocHost((void**)&ctx->h_pinned, (size_t)(3 * kMaxKrylov + 8) * sizeof(double)) != cudaSuccess) {
    ctx->err = "cudaMallocHost failed";
    return fail(RSC_ENOMEM);
  }
  *out = ctx;
  return RSC_OK;
}

rsc_status rsc_destroy(rsc_ctx* ctx) {
  if (!ctx) return RSC_EINVAL;
  if (ctx->s) cudaStreamSynchronize(ctx->s);
  else cudaDeviceSynchronize();
  if (ctx->jvp_exec) cudaGraphExecDestroy(ctx->jvp_exec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->s2) cudaStreamSynchronize(ctx->s2), cudaStreamDestroy(ctx->s2);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  void* bufs[] = {(void*)ctx->d_slots, ctx->d_cslot, ctx->jvp_y, ctx->tc_tiles, ctx->tc_off, ctx->tc_kpad, ctx->d_status, ctx->d_EcT1, ctx->d_m_of, ctx->d_pstart, ctx->d_pair_l, ctx->d_pair_m, ctx->d_leg_off,
                  ctx->d_rc, ctx->d_rd, ctx->d_EcT0, ctx->d_EcT2, ctx->d_EdT0, ctx->d_EdT1,
                  ctx->d_EdT2, ctx->d_R0T, ctx->d_R1T, ctx->f_EdT0, ctx->f_EdT1,
                  ctx->f_EdT2, ctx->f_R0T, ctx->f_R1T, ctx->f_rd, ctx->f_EcT0, ctx->f_EcT2, ctx->SR, ctx->FC, ctx->FCU, ctx->UG, ctx->FA,
                  ctx->AR, ctx->rhs, ctx->mid, ctx->xtmp, ctx->vtmp, ctx->rtmp, ctx->ustate, ctx->ref_tmp, ctx->d_Ef[0], ctx->d_Ef[1], ctx->d_Ef[2], ctx->d_Ef[3], ctx->V, ctx->Vs, ctx->partial,
                  ctx->dots, ctx->AR0, ctx->ta_tiles, ctx->ta_off, ctx->cont_hist, ctx->cont_cond, ctx->amax_v, ctx->amax_i, ctx->d_keT, ctx->d_kedT, ctx->d_ker, ctx->d_kew, ctx->d_diag, ctx->d_cr_pairs, ctx->d_E01, ctx->cr_w, ctx->d_cr_rowf, ctx->d_cr_pairf};
  for (void* b : bufs) cudaFree(b);
  for (int q = 0; q < 8; ++q) {
    cudaFree(ctx->leg64.buf[q]);
    cudaFree(ctx->leg32.buf[q]);
  }
  for (auto& f : ctx->fac) free_factor(f);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  drain_events(ctx);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  delete ctx;
  return RSC_OK;
}

rsc_status rsc_set_params(rsc_ctx* ctx, const rsc_params* params) {
  if (!ctx) return RSC_EINVAL;
  CKS(check_params(params));
  if (params->L != ctx->p.L || params->Ms != ctx->p.Ms || params->Nr != ctx->p.Nr ||
      params->precision != ctx->p.precision) {
    ctx->err = "L, Ms, Nr and precision are fixed for a context";
    return RSC_EINVAL;
  }
  const bool refactor = params->Ek != ctx->p.Ek || params->Pr != ctx->p.Pr ||
                        params->eta != ctx->p.eta ||
                        params->explicit_coriolis != ctx->p.explicit_coriolis;
  if (params->eta != ctx->p.eta) {
    ctx->err = "eta is fixed for a context (it defines the radial grid)";
    return RSC_EINVAL;
  }
  CK(cudaStreamSynchronize(ctx->s));
  ctx->p = *params;
  if (refactor) {
    for (auto& f : ctx->fac) free_factor(f);
    ctx->share.reset();   // another operator: this context factorises on its own
  }
  if (ctx->jvp_exec) {   // captured launches embed parameters and factor pointers
    cudaGraphExecDestroy(ctx->jvp_exec);
    ctx->jvp_exec = nullptr;
  }
  return RSC_OK;
}

rsc_status rsc_state_size(const rsc_ctx* ctx, size_t* n_real, int* n_pairs) {
  if (!ctx) return RSC_EINVAL;
  if (n_real) *n_real = (size_t)ctx->d.n();
  if (n_pairs) *n_pairs = ctx->d.P;
  return RSC_OK;
}

rsc_status rsc_conductive_state(rsc_ctx* ctx, double* U) {
  if (!ctx || !U) return RSC_EINVAL;
  std::vector<double> coef;
  conductive_T00(ctx->p, ctx->d, ctx->t, coef);
  const long n = ctx->d.n();
  CK(cudaMemsetAsync(U, 0, n * sizeof(double), ctx->s));
  // T_00 is pair 0 (m = 0, l = 0) of field 2; real parts at stride 2.
  std::vector<double> row(2 * ctx->d.Nr, 0.0);
  for (int k = 0; k < ctx->d.Nr; ++k) row[2 * k] = coef[k];
  double* dst = U + (long)2 * ctx->d.P * ctx->d.Nr * 2;
  CK(cudaMemcpyAsync(dst, row.data(), row.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  return RSC_OK;
}

rsc_status rsc_step(rsc_ctx* ctx, double* U, double C, double dt, int nsteps) {
  if (!ctx || !U || nsteps < 0 || !(dt > 0)) return RSC_EINVAL;
  const bool fp32 = ctx->p.precision == RSC_MIXED;
  for (int s = 0; s < nsteps; ++s) CKS(step_any(ctx, U, C, dt, fp32));
  return RSC_OK;
}

rsc_status rsc_step2(rsc_ctx* ctx, double* U, double dt, int nsteps) {
  if (!ctx || !U || nsteps < 0 || !(dt > 0)) return RSC_EINVAL;
  const bool fp32 = ctx->p.precision == RSC_MIXED;
  for (int s = 0; s < nsteps; ++s)
    CKS(fp32 ? do_step2<float>(ctx, U, dt) : do_step2<double>(ctx, U, dt));
  return RSC_OK;
}

rsc_status rsc_step_host(rsc_ctx* ctx, double* U_host, double C, double dt, int nsteps) {
  if (!ctx || !U_host) return RSC_EINVAL;
  const long n = ctx->d.n();
  CK(cudaMemcpyAsync(ctx->ustate, U_host, n * sizeof(double), cudaMemcpyHostToDevice, ctx->s));
  CKS(rsc_step(ctx, ctx->ustate, C, dt, nsteps));
  CK(cudaMemcpyAsync(U_host, ctx->ustate, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  return RSC_OK;
}

rsc_status rsc_explicit_terms(rsc_ctx* ctx, const double* U, double* N) {
  if (!ctx || !U || !N) return RSC_EINVAL;
  if (ctx->p.precision == RSC_MIXED) {
    CKS(stage_synth<float>(ctx, U, ctx->FC));
    CKS(stage_products_analysis<float>(ctx, false));
    CKS(stage_rhs<float>(ctx, make_rp(ctx, 1.0, 0.0, 2), U, nullptr, nullptr,
                         reinterpret_cast<double2*>(N)));
  } else {
    CKS(stage_synth<double>(ctx, U, ctx->FC));
    CKS(stage_products_analysis<double>(ctx, false));
    CKS(stage_rhs<double>(ctx, make_rp(ctx, 1.0, 0.0, 2), U, nullptr, nullptr,
                          reinterpret_cast<double2*>(N)));
  }
  return RSC_OK;
}

rsc_status rsc_apply_jacobian(rsc_ctx* ctx, const double* U, double C, long J, const double* u,
                              double* out, int count, double dt) {
  if (!ctx || !U || !u || !out || count < 0 || !(dt > 0)) return RSC_EINVAL;
  const long n = ctx->d.n();
  if (J >= n) return RSC_EINVAL;
  const bool fp32 = ctx->p.precision == RSC_MIXED;
  CKS(cache_base(ctx, U, fp32));
  for (int q = 0; q < count; ++q)
    CKS(jvp_any(ctx, U, C, J < 0 ? -1 : J, u + (long)q * n, out + (long)q * n, dt, fp32));
  return RSC_OK;
}

static const char* kKernelNames[RSC_NUM_KERNELS] = {
    "radial_eval", "legendre_synth", "fft_products", "legendre_analysis", "rhs_assemble",
    "chain_solve", "temp_solve", "gmres_dots", "gmres_axpy", "blas1", "chain_sweep",
    "chain_reduced"};

const char* rsc_kernel_name(int id) {
  return (id >= 0 && id < RSC_NUM_KERNELS) ? kKernelNames[id] : "unknown";
}

rsc_status rsc_profile_enable(rsc_ctx* ctx, int on) {
  if (!ctx) return RSC_EINVAL;
  drain_events(ctx);
  for (int k = 0; k < RSC_NUM_KERNELS; ++k) {
    ctx->prof_ms[k] = 0.0;
    ctx->prof_launches[k] = 0;
    ctx->prof_bytes[k] = 0.0;
    ctx->prof_flops[k] = 0.0;
  }
  ctx->prof_on = on != 0;
  ctx->prof_mask = (unsigned)on;
  return RSC_OK;
}

rsc_status rsc_profile_query(rsc_ctx* ctx, int id, double* ms, long* launches, double* bytes,
                             double* flops) {
  if (!ctx || id < 0 || id >= RSC_NUM_KERNELS) return RSC_EINVAL;
  drain_events(ctx);
  if (ms) *ms = ctx->prof_ms[id];
  if (launches) *launches = ctx->prof_launches[id];
  if (bytes) *bytes = ctx->prof_bytes[id];
  if (flops) *flops = ctx->prof_flops[id];
  return RSC_OK;
}

rsc_status rsc_launch_count(const rsc_ctx* ctx, long* count) {
  if (!ctx || !count) return RSC_EINVAL;
  *count = ctx->launches;
  return RSC_OK;
}

rsc_status rsc_norm2(rsc_ctx* ctx, const double* v, size_t n, double* out) {
  if (!ctx || !v || !out) return RSC_EINVAL;
  return norm2(ctx, v, (long)n, out);
}

rsc_status rsc_diagnostics(rsc_ctx* ctx, const double* U, double* KE, double* Nu_in,
                           double* Nu_out) {
  if (!ctx || !U) return RSC_EINVAL;
  double v[3];
  CKS(diagnostics(ctx, U, v));
  if (KE) *KE = v[0];
  if (Nu_in) *Nu_in = v[1];
  if (Nu_out) *Nu_out = v[2];
  return RSC_OK;
}

rsc_status rsc_newton_rw(rsc_ctx* ctx, double* U, double* C, long J, const rsc_newton_opts* o,
                         rsc_newton_report* rep) {
  if (!ctx || !U || !C || !o) return RSC_EINVAL;
  if (o->kmax < 1 || o->kmax > kMaxKrylov || o->max_newton < 0 || !(o->dt_newton > 0))
    return RSC_EINVAL;
  const long n = ctx->d.n();
  if (J >= n) return RSC_EINVAL;
  const auto t0 = std::chrono::steady_clock::now();
  rsc_newton_report local{};
  rsc_newton_report* r = rep ? rep : &local;
  std::memset(r, 0, sizeof(*r));
  const bool fp32 = ctx->p.precision == RSC_MIXED;
  int nb;
  launch_1d_grid(n, &nb);
  double Cv = *C;
  rsc_status result = RSC_ENOCONV;
  for (int it = 0; it <= o->max_newton; ++it) {
    // residual B(U) - U in FP64 (the refinement step of the mixed path)
    CK(cudaMemcpyAsync(ctx->rtmp, U, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->s));
    CKS(step_any(ctx, ctx->rtmp, Cv, o->dt_newton, false));
    {
      KSpan sp(ctx, RSC_K_BLAS, 24.0 * n, 2.0 * n);
      k_axpby<<<nb, 256, 0, ctx->s>>>(-1.0, U, 1.0, ctx->rtmp, n);
      CK(cudaGetLastError());
    }
    double rn;
    CKS(norm2(ctx, ctx->rtmp, n, &rn));
    CKS(check_status(ctx));
    if (it < RSC_MAX_HISTORY) r->residual_history[it] = rn;
    r->residual = rn;
    r->iterations = it;
    if (!std::isfinite(rn)) {
      ctx->err = "non-finite Newton residual";
      result = RSC_ENAN;
      break;
    }
    if (rn < o->tol) {
      result = RSC_OK;
      break;
    }
    if (it == o->max_newton) break;
    CKS(cache_base(ctx, U, fp32));
    int its = 0;
    double rel = 0;
    CKS(gmres(ctx, U, Cv, J < 0 ? -1 : J, ctx->rtmp, ctx->vtmp, o->dt_newton, o->kmax,
              o->gmres_tol, fp32, &its, &rel));
    if (it < RSC_MAX_HISTORY) r->gmres_history[it] = its;
    r->gmres_total += its;
    double c = 0.0;
    if (J >= 0) {
      CK(cudaMemcpyAsync(ctx->h_pinned, ctx->vtmp + J, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
      CK(cudaStreamSynchronize(ctx->s));
      c = ctx->h_pinned[0];
      CK(cudaMemsetAsync(ctx->vtmp + J, 0, sizeof(double), ctx->s));
    }
    {
      KSpan sp(ctx, RSC_K_BLAS, 24.0 * n, 2.0 * n);
      k_axpby<<<nb, 256, 0, ctx->s>>>(-1.0, ctx->vtmp, 1.0, U, n);
      CK(cudaGetLastError());
    }
    Cv -= c;
  }
  CK(cudaStreamSynchronize(ctx->s));
  *C = Cv;
  r->C = Cv;
  r->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (result == RSC_ENOCONV) ctx->err = "Newton iteration cap reached";
  return result;
}

rsc_status rsc_newton_rw_host(rsc_ctx* ctx, double* U_host, double* C, long J,
                              const rsc_newton_opts* o, rsc_newton_report* rep) {
  if (!ctx || !U_host || !C) return RSC_EINVAL;
  const long n = ctx->d.n();
  // the device copy lives in a buffer the context allocated at creation
  CK(cudaMemcpyAsync(ctx->ustate, U_host, n * sizeof(double), cudaMemcpyHostToDevice, ctx->s));
  const rsc_status st = rsc_newton_rw(ctx, ctx->ustate, C, J, o, rep);
  if (st != RSC_OK && st != RSC_ENOCONV) return st;
  CK(cudaMemcpyAsync(U_host, ctx->ustate, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  return st;
}

rsc_status rsc_factor_block(rsc_ctx* ctx, double dt, int which, long index, double* out_host) {
  if (!ctx || !out_host || which < 0 || which > 7 || index < 0 || !(dt > 0) || !std::isfinite(dt))
    return RSC_EINVAL;
  const Dims& d = ctx->d;
  const size_t blk = (size_t)d.Nr * d.Nr;
  long nblk = 0, nodd = 0;
  for (int a = 0; a < d.nm; ++a) {
    nblk += 2L * (d.L - ctx->t.m_of[a] + 1);
    nodd += 2L * ((d.L - ctx->t.m_of[a] + 1) / 2);
  }
  if ((which < 3 && index >= nblk) || (which == 3 && index > d.L) ||
      (which == 4 && index >= nodd) || (which > 4 && index >= nblk - nodd))
    return RSC_EINVAL;
  if (which >= 4 && (ctx->p.precision != RSC_MIXED || ctx->p.explicit_coriolis ||
                     ctx->chain_parts != 1)) {
    ctx->err = "reduced-chain factors exist on mixed contexts with implicit Coriolis only";
    return RSC_EINVAL;
  }
  DevFactor* f = nullptr;
  CKS(get_factor(ctx, dt, &f));
  if (which >= 4) {
    CKS(ensure_cr_locked(ctx, f));
    const float4* src = which == 4 ? f->Ds : which == 5 ? f->Gr : which == 6 ? f->Hr : f->Wr;
    std::vector<float4> t(blk);
    CK(cudaMemcpyAsync(t.data(), src + index * blk, blk * sizeof(float4), cudaMemcpyDeviceToHost,
                       ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    for (size_t e = 0; e < blk; ++e) {
      out_host[2 * e] = (double)t[e].x + (double)t[e].z;
      out_host[2 * e + 1] = (double)t[e].y + (double)t[e].w;
    }
    return RSC_OK;
  }
  if (which == 3)
    CK(cudaMemcpyAsync(out_host, f->Tinv + index * blk, blk * sizeof(double),
                       cudaMemcpyDeviceToHost, ctx->s));
  else {
    const double2* src = which == 0 ? f->G : which == 1 ? f->H : f->W;
    CK(cudaMemcpyAsync(out_host, src + index * blk, blk * sizeof(double2), cudaMemcpyDeviceToHost,
                       ctx->s));
  }
  CK(cudaStreamSynchronize(ctx->s));
  return RSC_OK;
}

rsc_status rsc_factor_time(const rsc_ctx* ctx, double* seconds, int* on_gpu) {
  if (!ctx) return RSC_EINVAL;
  if (seconds) *seconds = ctx->factor_s;
  if (on_gpu) *on_gpu = ctx->factor_on_gpu;
  return RSC_OK;
}

rsc_status rsc_factor_time_cr(const rsc_ctx* ctx, double* seconds, int* on_gpu) {
  if (!ctx) return RSC_EINVAL;
  if (seconds) *seconds = ctx->factor_cr_s;
  if (on_gpu) *on_gpu = ctx->factor_cr_on_gpu;
  return RSC_OK;
}

rsc_status rsc_implicit_solve(rsc_ctx* ctx, const double* rhs, double* x, double dt) {
  if (!ctx || !rhs || !x || !(dt > 0) || !std::isfinite(dt)) return RSC_EINVAL;
  DevFactor* f = nullptr;
  CKS(get_factor(ctx, dt, &f));
  CK(cudaMemcpyAsync(ctx->rhs, rhs, (size_t)ctx->d.n() * sizeof(double), cudaMemcpyDeviceToDevice,
                     ctx->s));
  if (ctx->p.precision == RSC_MIXED)
    CKS(stage_solve(ctx, f, x, true));
  else
    CKS(stage_solve_fp64(ctx, f, x));
  return RSC_OK;
}

rsc_status rsc_autotune(rsc_ctx* ctx, rsc_tuning* out) {
  if (!ctx) return RSC_EINVAL;
  return autotune(ctx, out);
}

rsc_status rsc_get_tuning(const rsc_ctx* ctx, rsc_tuning* out) {
  if (!ctx || !out) return RSC_EINVAL;
  get_tuning(ctx, out);
  return RSC_OK;
}

rsc_status rsc_set_tuning(rsc_ctx* ctx, const rsc_tuning* t) {
  if (!ctx || !t) return RSC_EINVAL;
  if (!tuning_ok(ctx, *t)) {
    ctx->err = "launch shapes not feasible for this context";
    return RSC_EINVAL;
  }
  CK(cudaStreamSynchronize(ctx->s));
  set_tuning(ctx, *t);
  return RSC_OK;
}

rsc_status rsc_continuation_predict(const double* Ra, const double* s, int npts, int n_its,
                                    int n_opt, double gamma, double alpha_scale, int* mode,
                                    double* Ra_new, double* w) {
  if (!Ra || !s || !mode || !Ra_new || !w || npts < 2) return RSC_EINVAL;
  const int k = npts < 3 ? npts : 3;
  const double alpha = alpha_scale * (n_opt + 1.0) / (n_its + 1.0);
  const double dRa = (Ra[0] - Ra[1]) / Ra[0];
  const double ds = s[0] != 0.0 ? (s[0] - s[1]) / s[0] : 0.0;
  *mode = std::fabs(ds) > gamma * std::fabs(dRa) ? 1 : 0;
  const double* nodes = *mode == 0 ? Ra : s;
  const double x = nodes[0] + alpha * (nodes[0] - nodes[1]);
  for (int p = 0; p < 3; ++p) {
    double v = 0.0;
    if (p < k) {
      v = 1.0;
      for (int q = 0; q < k; ++q)
        if (q != p) v *= (x - nodes[q]) / (nodes[p] - nodes[q]);
    }
    w[p] = v;
  }
  if (*mode == 0) {
    *Ra_new = x;
  } else {
    double r = 0.0;
    for (int p = 0; p < k; ++p) r += w[p] * Ra[p];
    *Ra_new = r;
  }
  return RSC_OK;
}

}  // extern "C"

namespace {

// One branch of a natural-parameter continuation (Sec. 4.3; Sec. 4.4 with x = log10 Ek):
// Newton solves at x0, x1, then predicted points until x passes x_end, max_points is
// reached, a step fails after all retries (RSC_ENOCONV) or, when tail_threshold > 0, a
// converged point's spectral tail exceeds it (RSC_ERESOLUTION).  set_x applies x to the
// context.  U returns the last converged state and *C its drift.
struct BranchPoint {
  double x, C, KE, Nu_in, Nu_out, residual, cheb_tail, sh_tail;
  int its, gmres, mode;
};

rsc_status spectral_tail(rsc_ctx* ctx, const double* U, double* cheb, double* sh);

template <typename SetX>
rsc_status follow_branch(rsc_ctx* ctx, double* U, double* C, long J, double x0, double x1,
                         double x_end, int n_opt, double gamma, int max_points, int retries,
                         double tail_threshold, const rsc_newton_opts* nopts, SetX set_x,
                         std::vector<BranchPoint>& pts) {
  const long n = ctx->d.n();
  int nb;
  launch_1d_grid(n, &nb);
  if (!ctx->cont_hist) {
    CK(cudaMalloc((void**)&ctx->cont_hist, 3 * (size_t)n * sizeof(double)));
    CK(cudaMalloc((void**)&ctx->cont_cond, (size_t)n * sizeof(double)));
    CK(cudaMalloc((void**)&ctx->amax_v, 1024 * sizeof(double)));
    CK(cudaMalloc((void**)&ctx->amax_i, 1025 * sizeof(long)));
  }
  CKS(rsc_conductive_state(ctx, ctx->cont_cond));
  double* H[3] = {ctx->cont_hist, ctx->cont_hist + n, ctx->cont_hist + 2 * n};
  int slot[3] = {-1, -1, -1};   // history slots, most recent first
  double hx[3] = {0, 0, 0}, hC[3] = {0, 0, 0};
  int last_its = 0;
  bool under = false;
  auto solve = [&](double x, double* Cv, BranchPoint* pt) -> bool {
    if (set_x(x) != RSC_OK) return false;
    rsc_newton_report rep{};
    if (rsc_newton_rw(ctx, U, Cv, J, nopts, &rep) != RSC_OK) return false;
    pt->x = x;
    pt->C = *Cv;
    pt->residual = rep.residual;
    pt->its = rep.iterations;
    pt->gmres = rep.gmres_total;
    double dg[3];
    if (diagnostics(ctx, U, dg) != RSC_OK) return false;
    pt->KE = dg[0];
    pt->Nu_in = dg[1];
    pt->Nu_out = dg[2];
    if (spectral_tail(ctx, U, &pt->cheb_tail, &pt->sh_tail) != RSC_OK) return false;
    return true;
  };
  auto push = [&](const BranchPoint& pt) -> rsc_status {
    const int fresh = slot[2] >= 0 ? slot[2] : (slot[1] >= 0 ? 2 : (slot[0] >= 0 ? 1 : 0));
    CK(cudaMemcpyAsync(H[fresh], U, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->s));
    slot[2] = slot[1]; slot[1] = slot[0]; slot[0] = fresh;
    hx[2] = hx[1]; hx[1] = hx[0]; hx[0] = pt.x;
    hC[2] = hC[1]; hC[1] = hC[0]; hC[0] = pt.C;
    last_its = pt.its;
    pts.push_back(pt);
    if (tail_threshold > 0 && std::max(pt.cheb_tail, pt.sh_tail) > tail_threshold) under = true;
    return RSC_OK;
  };
  rsc_status result = RSC_OK;
  double Cv = *C;
  BranchPoint pt{};
  if (!solve(x0, &Cv, &pt)) {
    ctx->err = "Newton did not converge at the first continuation point";
    return RSC_ENOCONV;
  }
  pt.mode = 0;
  CKS(push(pt));
  if (!under) {
    if (!solve(x1, &Cv, &pt)) {
      result = RSC_ENOCONV;
    } else {
      pt.mode = 0;
      CKS(push(pt));
    }
  }
  const double dir = x1 > x0 ? 1.0 : -1.0;
  while (result == RSC_OK && !under && (int)pts.size() < max_points &&
         dir * (pts.back().x - x_end) < 0) {
    const int k = pts.size() < 3 ? (int)pts.size() : 3;
    // J of the last point: the largest |U - U_cond|
    {
      KSpan sp(ctx, RSC_K_BLAS, 16.0 * n, 1.0 * n);
      k_argmax_absdiff<<<nb, 256, 0, ctx->s>>>(H[slot[0]], ctx->cont_cond, n, ctx->amax_v,
                                               ctx->amax_i);
      CK(cudaGetLastError());
    }
    {
      KSpan sp(ctx, RSC_K_BLAS, 16.0 * nb, 1.0 * nb);
      k_argmax_finish<<<1, 256, 0, ctx->s>>>(ctx->amax_v, ctx->amax_i, nb, ctx->amax_i + 1024);
      CK(cudaGetLastError());
    }
    long jm = 0;
    CK(cudaMemcpyAsync(&jm, ctx->amax_i + 1024, sizeof(long), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    double sv[3] = {0, 0, 0}, uc = 0.0;
    CK(cudaMemcpy(&uc, ctx->cont_cond + jm, sizeof(double), cudaMemcpyDeviceToHost));
    for (int q = 0; q < k; ++q) {
      CK(cudaMemcpy(&sv[q], H[slot[q]] + jm, sizeof(double), cudaMemcpyDeviceToHost));
      sv[q] -= uc;
    }
    bool ok = false;
    for (int attempt = 0; attempt <= retries && !ok; ++attempt) {
      int mode = 0;
      double x_new = 0.0, w[3];
      CKS(rsc_continuation_predict(hx, sv, k, last_its, n_opt, gamma, std::ldexp(1.0, -attempt),
                                   &mode, &x_new, w));
      {
        KSpan sp(ctx, RSC_K_BLAS, 8.0 * n * (k + 1), 2.0 * n * k);
        k_lincomb3<<<nb, 256, 0, ctx->s>>>(U, w[0], H[slot[0]], w[1], H[slot[1]], w[2],
                                           k > 2 ? H[slot[2]] : nullptr, n);
        CK(cudaGetLastError());
      }
      Cv = w[0] * hC[0] + w[1] * hC[1] + (k > 2 ? w[2] * hC[2] : 0.0);
      if (solve(x_new, &Cv, &pt)) {
        pt.mode = mode;
        CKS(push(pt));
        ok = true;
      }
    }
    if (!ok) result = RSC_ENOCONV;
  }
  // leave the last converged state in U and the context at its parameter
  CK(cudaMemcpyAsync(U, H[slot[0]], n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  CKS(set_x(hx[0]));
  *C = hC[0];
  if (result == RSC_ENOCONV) ctx->err = "a continuation step did not converge after all retries";
  if (result == RSC_OK && under) {
    ctx->err = "the last point is under-resolved (spectral tail above the threshold)";
    result = RSC_ERESOLUTION;
  }
  return result;
}

rsc_status spectral_tail(rsc_ctx* ctx, const double* U, double* cheb, double* sh) {
  const Dims& d = ctx->d;
  const long n = d.n();
  if (!ctx->cont_cond) CK(cudaMalloc((void**)&ctx->cont_cond, (size_t)n * sizeof(double)));
  if (!ctx->amax_v) CK(cudaMalloc((void**)&ctx->amax_v, 1024 * sizeof(double)));
  if (!ctx->amax_i) CK(cudaMalloc((void**)&ctx->amax_i, 1025 * sizeof(long)));
  CKS(rsc_conductive_state(ctx, ctx->cont_cond));
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(ctx->amax_v);
  CK(cudaMemsetAsync(acc, 0, 3 * sizeof(unsigned long long), ctx->s));
  int nb;
  launch_1d_grid(n / 2, &nb);
  {
    KSpan sp(ctx, RSC_K_BLAS, 16.0 * n, 4.0 * n);
    k_spectral_tail<<<nb, 256, 0, ctx->s>>>(reinterpret_cast<const double2*>(U),
                                            reinterpret_cast<const double2*>(ctx->cont_cond),
                                            d.P, d.Nr, d.L, ctx->d_pair_l, acc);
    CK(cudaGetLastError());
  }
  unsigned long long h[3];
  CK(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  double v[3];
  std::memcpy(v, h, sizeof(v));
  *cheb = v[0] > 0 ? v[1] / v[0] : 0.0;
  *sh = v[0] > 0 ? v[2] / v[0] : 0.0;
  return RSC_OK;
}

}  // namespace

extern "C" {

rsc_status rsc_continue_ra(rsc_ctx* ctx, double* U, double* C, long J,
                           const rsc_continuation_opts* o, rsc_continuation_point* pts,
                           int* npoints) {
  if (!ctx || !U || !C || !o || !pts || !npoints || o->max_points < 2 || o->retries < 0 ||
      !(o->Ra0 > 0) || !(o->Ra1 > 0) || o->Ra0 == o->Ra1)
    return RSC_EINVAL;
  *npoints = 0;
  auto set_ra = [&](double Ra) -> rsc_status {
    rsc_params q = ctx->p;     // Ra enters only the explicit terms: no refactorisation
    q.Ra = Ra;
    return rsc_set_params(ctx, &q);
  };
  std::vector<BranchPoint> bp;
  const rsc_status st = follow_branch(ctx, U, C, J, o->Ra0, o->Ra1, o->Ra_end, o->n_opt, o->gamma,
                                      o->max_points, o->retries, 0.0, &o->newton, set_ra, bp);
  for (const BranchPoint& b : bp) {
    rsc_continuation_point& q = pts[(*npoints)++];
    q.Ra = b.x; q.C = b.C; q.KE = b.KE; q.Nu_in = b.Nu_in; q.Nu_out = b.Nu_out;
    q.residual = b.residual; q.newton_iterations = b.its; q.gmres_total = b.gmres; q.mode = b.mode;
  }
  return st;
}

rsc_status rsc_continue_ek(rsc_ctx* ctx, double* U, double* C, long J,
                           const rsc_ek_continuation_opts* o, rsc_ek_point* pts, int* npoints) {
  if (!ctx || !U || !C || !o || !pts || !npoints || o->max_points < 2 || o->retries < 0 ||
      !(o->Ek0 > 0) || !(o->Ek1 > 0) || !(o->Ek_end > 0) || o->Ek0 == o->Ek1 || o->ra_coef < 0)
    return RSC_EINVAL;
  *npoints = 0;
  // x = log10 Ek (Eq. new_EK); Ek enters the implicit operator, so every new value refactorises
  auto set_ek = [&](double x) -> rsc_status {
    rsc_params q = ctx->p;
    q.Ek = std::pow(10.0, x);
    if (o->ra_coef > 0) q.Ra = o->ra_coef * std::pow(q.Ek, -1.0 / 3.0);
    if (q.Ek == ctx->p.Ek && q.Ra == ctx->p.Ra) return RSC_OK;
    return rsc_set_params(ctx, &q);
  };
  std::vector<BranchPoint> bp;
  const rsc_status st = follow_branch(ctx, U, C, J, std::log10(o->Ek0), std::log10(o->Ek1),
                                      std::log10(o->Ek_end), o->n_opt, o->gamma, o->max_points,
                                      o->retries, o->tail_threshold, &o->newton, set_ek, bp);
  for (const BranchPoint& b : bp) {
    rsc_ek_point& q = pts[(*npoints)++];
    q.Ek = std::pow(10.0, b.x);
    q.Ra = o->ra_coef > 0 ? o->ra_coef * std::pow(q.Ek, -1.0 / 3.0) : ctx->p.Ra;
    q.C = b.C; q.KE = b.KE; q.Nu_in = b.Nu_in; q.Nu_out = b.Nu_out; q.residual = b.residual;
    q.cheb_tail = b.cheb_tail; q.sh_tail = b.sh_tail;
    q.newton_iterations = b.its; q.gmres_total = b.gmres; q.mode = b.mode;
  }
  return st;
}

rsc_status rsc_spectral_tail(rsc_ctx* ctx, const double* U, double* cheb, double* sh) {
  if (!ctx || !U || !cheb || !sh) return RSC_EINVAL;
  return spectral_tail(ctx, U, cheb, sh);
}

rsc_status rsc_regrid(const rsc_ctx* src, const double* U_src, rsc_ctx* dst, double* U_dst) {
  if (!src || !dst || !U_src || !U_dst) return RSC_EINVAL;
  if (src->d.Ms != dst->d.Ms || src->p.eta != dst->p.eta) {
    dst->err = "regrid needs the same azimuthal symmetry and radius ratio";
    return RSC_EINVAL;
  }
  rsc_ctx* ctx = dst;
  const long n = dst->d.n();
  int nb;
  launch_1d_grid(n / 2, &nb);
  {
    KSpan sp(ctx, RSC_K_BLAS, 16.0 * n, 0.0);
    k_regrid<<<nb, 256, 0, dst->s>>>(reinterpret_cast<const double2*>(U_src), src->d.L, src->d.Nr,
                                     src->d.P, reinterpret_cast<double2*>(U_dst), dst->d.Nr,
                                     dst->d.P, dst->d_pair_l, dst->d_pair_m, dst->d.Ms);
    CK(cudaGetLastError());
  }
  return RSC_OK;
}

rsc_status rsc_refine_params(const rsc_params* p, double cheb_tail, double sh_tail,
                             double threshold, double growth, rsc_params* out, int* refined) {
  if (!p || !out || !refined || !(growth > 1.0) || !(threshold > 0)) return RSC_EINVAL;
  *out = *p;
  *refined = 0;
  if (cheb_tail > threshold) {
    out->Nr = std::min(128, (int)std::ceil(p->Nr * growth));
    if (out->Nr > p->Nr) *refined |= 1;
  }
  if (sh_tail > threshold) {
    out->L = std::min(255, (int)std::ceil(p->L * growth));
    if (out->L > p->L) *refined |= 2;
  }
  return RSC_OK;
}

// ===========================================================================
// Batches of instances (continuation points in Ra, waves of different azimuthal
// symmetries): one context per instance on its own stream; batched Jacobian actions
// are captured into one CUDA graph whose branches run the instances concurrently.
}  // extern "C"

struct rsc_batch {
  std::vector<rsc_ctx*> ctx;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaStream_t s = nullptr;          // the caller's stream (graph launches)
  cudaGraphExec_t exec = nullptr;
  long nodes = 0;
  // key of the captured graph
  std::vector<const double*> kU, ku;
  std::vector<double*> kout;
  std::vector<double> kC;
  std::vector<long> kJ;
  int kcount = -1;
  double kdt = 0;
  std::string err;
};

namespace {
void batch_free(rsc_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (rsc_ctx* c : b->ctx)
    if (c) rsc_destroy(c);
  for (cudaStream_t st : b->streams) cudaStreamDestroy(st);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}
}  // namespace

extern "C" {

rsc_status rsc_batch_create(const rsc_params* params, int n, void* stream, rsc_batch** out) {
  if (!params || !out || n < 1 || n > 4096) return RSC_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i) CKS(check_params(&params[i]));
  rsc_batch* b = new (std::nothrow) rsc_batch();
  if (!b) return RSC_ENOMEM;
  b->s = reinterpret_cast<cudaStream_t>(stream);
  b->ctx.assign(n, nullptr);
  b->streams.assign(n, nullptr);
  b->join.assign(n, nullptr);
  rsc_status st = RSC_OK;
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) st = RSC_ECUDA;
  for (int i = 0; i < n && st == RSC_OK; ++i) {
    if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) != cudaSuccess) {
      st = RSC_ECUDA;
      break;
    }
    st = rsc_create(&params[i], b->streams[i], &b->ctx[i]);
    if (st != RSC_OK) b->err = "instance " + std::to_string(i) + ": " + rsc_last_error(b->ctx[i]);
  }
  if (st != RSC_OK) {
    batch_free(b);
    return st;
  }
  // instances with the same operator share one set of factorisations
  auto same_operator = [&](const rsc_params& a, const rsc_params& c) {
    return a.L == c.L && a.Ms == c.Ms && a.Nr == c.Nr && a.Ek == c.Ek && a.Pr == c.Pr &&
           a.eta == c.eta && a.precision == c.precision &&
           a.explicit_coriolis == c.explicit_coriolis;
  };
  for (int i = 0; i < n; ++i) {
    if (b->ctx[i]->share) continue;
    std::shared_ptr<FactorShare> sh;
    for (int j = i + 1; j < n; ++j)
      if (!b->ctx[j]->share && same_operator(params[i], params[j])) {
        if (!sh) {
          sh = std::make_shared<FactorShare>();
          b->ctx[i]->share = sh;
        }
        b->ctx[j]->share = sh;
      }
  }
  *out = b;
  return RSC_OK;
}

rsc_status rsc_batch_destroy(rsc_batch* b) {
  if (!b) return RSC_EINVAL;
  if (b->s) cudaStreamSynchronize(b->s);
  for (cudaStream_t st : b->streams) cudaStreamSynchronize(st);
  batch_free(b);
  return RSC_OK;
}

rsc_status rsc_batch_size(const rsc_batch* b, int* n) {
  if (!b || !n) return RSC_EINVAL;
  *n = (int)b->ctx.size();
  return RSC_OK;
}

rsc_status rsc_batch_context(rsc_batch* b, int i, rsc_ctx** ctx) {
  if (!b || !ctx || i < 0 || i >= (int)b->ctx.size()) return RSC_EINVAL;
  *ctx = b->ctx[i];
  return RSC_OK;
}

const char* rsc_batch_last_error(const rsc_batch* b) { return b ? b->err.c_str() : "null batch"; }

rsc_status rsc_batch_apply_jacobian(rsc_batch* b, const double* const* U, const double* C,
                                    const long* J, const double* const* u, double* const* out,
                                    int count, double dt) {
  if (!b || !U || !C || !J || !u || !out || count < 1 || !(dt > 0)) return RSC_EINVAL;
  const int n = (int)b->ctx.size();
  for (int i = 0; i < n; ++i)
    if (!U[i] || !u[i] || !out[i] || J[i] >= b->ctx[i]->d.n()) return RSC_EINVAL;
  bool same = b->exec && b->kcount == count && b->kdt == dt;
  for (int i = 0; i < n && same; ++i)
    same = b->kU[i] == U[i] && b->ku[i] == u[i] && b->kout[i] == out[i] && b->kC[i] == C[i] &&
           b->kJ[i] == J[i];
  auto fail = [&](rsc_status st, const std::string& what) {
    b->err = what;
    return st;
  };
  if (!same) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    // factorisations first: nothing may allocate or copy synchronously during capture
    for (int i = 0; i < n; ++i) {
      DevFactor* f = nullptr;
      if (get_factor(b->ctx[i], dt, &f) != RSC_OK || cudaStreamSynchronize(b->streams[i]) != cudaSuccess)
        return fail(RSC_ECUDA, "instance " + std::to_string(i) + ": " + b->ctx[i]->err);
    }
    cudaStream_t origin = b->s;
    cudaStream_t own = nullptr;
    if (!origin) {   // the legacy stream cannot be captured: use a private one
      if (cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess)
        return fail(RSC_ECUDA, "stream creation failed");
      origin = own;
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return fail(RSC_ECUDA, "cudaStreamBeginCapture failed");
    rsc_status st = RSC_OK;
    long nodes = 0;
    if (cudaEventRecord(b->fork, origin) != cudaSuccess) st = RSC_ECUDA;
    for (int i = 0; i < n && st == RSC_OK; ++i) {
      rsc_ctx* c = b->ctx[i];
      if (cudaStreamWaitEvent(b->streams[i], b->fork, 0) != cudaSuccess) { st = RSC_ECUDA; break; }
      const bool prof = c->prof_on;
      c->prof_on = false;
      const long before = c->launches;
      const bool fp32 = c->p.precision == RSC_MIXED;
      DevFactor* f = nullptr;
      st = get_factor(c, dt, &f);
      if (st == RSC_OK) st = cache_base(c, U[i], fp32);
      const long nn = c->d.n();
      for (int q = 0; q < count && st == RSC_OK; ++q) {
        const long Jq = J[i] < 0 ? -1 : J[i];
        st = fp32 ? do_jvp_eager<float>(c, U[i], C[i], Jq, u[i] + q * nn, out[i] + q * nn, f, dt)
                  : do_jvp_eager<double>(c, U[i], C[i], Jq, u[i] + q * nn, out[i] + q * nn, f, dt);
      }
      nodes += c->launches - before;
      c->prof_on = prof;
      if (st == RSC_OK && (cudaEventRecord(b->join[i], b->streams[i]) != cudaSuccess ||
                           cudaStreamWaitEvent(origin, b->join[i], 0) != cudaSuccess))
        st = RSC_ECUDA;
      if (st != RSC_OK) b->err = "instance " + std::to_string(i) + ": " + c->err;
    }
    const cudaError_t ce = cudaStreamEndCapture(origin, &graph);
    if (st == RSC_OK && ce != cudaSuccess) st = fail(RSC_ECUDA, cudaGetErrorString(ce));
    if (st == RSC_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess)
      st = fail(RSC_ECUDA, "cudaGraphInstantiate failed");
    if (graph) cudaGraphDestroy(graph);
    if (own) cudaStreamDestroy(own);
    if (st != RSC_OK) {
      b->exec = nullptr;
      return st;
    }
    b->nodes = nodes;
    b->kU.assign(U, U + n);
    b->ku.assign(u, u + n);
    b->kout.assign(out, out + n);
    b->kC.assign(C, C + n);
    b->kJ.assign(J, J + n);
    b->kcount = count;
    b->kdt = dt;
  }
  cudaStream_t origin = b->s;
  if (cudaGraphLaunch(b->exec, origin) != cudaSuccess)
    return fail(RSC_ECUDA, "cudaGraphLaunch failed");
  for (rsc_ctx* c : b->ctx) c->launches += b->nodes / n;
  return RSC_OK;
}

rsc_status rsc_batch_autotune(rsc_batch* b) {
  if (!b) return RSC_EINVAL;
  const int n = (int)b->ctx.size();
  for (int i = 0; i < n; ++i) {
    const rsc_params& p = b->ctx[i]->p;
    int src = -1;   // an earlier instance with the same shape
    for (int j = 0; j < i && src < 0; ++j) {
      const rsc_params& q = b->ctx[j]->p;
      if (q.L == p.L && q.Ms == p.Ms && q.Nr == p.Nr && q.precision == p.precision &&
          q.Ek == p.Ek && q.Pr == p.Pr && q.explicit_coriolis == p.explicit_coriolis)
        src = j;
    }
    rsc_tuning t{};
    rsc_status st = src < 0 ? rsc_autotune(b->ctx[i], &t) : rsc_get_tuning(b->ctx[src], &t);
    if (st == RSC_OK && src >= 0) st = rsc_set_tuning(b->ctx[i], &t);
    if (st != RSC_OK) {
      b->err = "instance " + std::to_string(i) + ": " + b->ctx[i]->err;
      return st;
    }
  }
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return RSC_OK;
}

rsc_status rsc_batch_newton_rw(rsc_batch* b, double* const* U, double* C, const long* J,
                               const rsc_newton_opts* opts, rsc_newton_report* reports,
                               rsc_status* status) {
  if (!b || !U || !C || !J || !opts || !status) return RSC_EINVAL;
  const int n = (int)b->ctx.size();
  if (b->s) cudaStreamSynchronize(b->s);
  std::vector<std::thread> th;
  th.reserve(n);
  for (int i = 0; i < n; ++i)
    th.emplace_back([&, i] {
      status[i] = rsc_newton_rw(b->ctx[i], U[i], &C[i], J[i], opts, reports ? &reports[i] : nullptr);
    });
  for (auto& t : th) t.join();
  rsc_status worst = RSC_OK;
  for (int i = 0; i < n; ++i)
    if (status[i] != RSC_OK && status[i] != RSC_ENOCONV) worst = status[i];
  if (worst != RSC_OK) return worst;
  for (int i = 0; i < n; ++i)
    if (status[i] == RSC_ENOCONV) return RSC_ENOCONV;
  return RSC_OK;
}

}  // extern "C"
