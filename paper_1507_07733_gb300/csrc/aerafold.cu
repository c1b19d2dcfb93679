// aerafold.cu -- host side of the C ABI in include/aerafold.h.
//
// The context owns: device copies of VEL tables (uploaded once, Sec. 3 of arXiv 1507.07733),
// per-trace-length twiddle tables (computed once on the host in FP64), per-(length, rate,
// pattern) frequency-cell tables, a workspace arena for the station spectra (the paper's
// shared static device buffers of Sec. 4, kept resident here), and a device error word.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/aerafold.h"
#include "kernels.cuh"
#include "tc_dft.cuh"

using namespace aerafold;

namespace {

// An NVTX range for profilers (Nsight Systems, ncu --nvtx) around each entry point's host
// work and launches and around the server's steps; no cost without a profiler attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr double kBandLoHz = 30e6;
constexpr double kBandHiHz = 80e6;
constexpr double kCMPerNs = 0.299792458;

struct PatternDev {
  ar_pattern_desc desc;
  float2* table = nullptr;
  size_t bytes = 0;
};

struct LenTables {
  float2* t1 = nullptr;    // [4][Q][P]
  float2* wn = nullptr;    // [N]
};

struct KernelCfg {
  size_t smem = 0;
  int grid = 0;
  int slab_direct = 0;   // corner slabs read from L2 (when staging them would cost occupancy)
};

// the message ar_last_error(NULL) returns: the last failing ar_create or ar_unfold_noalloc of
// the calling thread (one per thread, so a failure on another thread never rewrites it)
thread_local std::string g_create_error;

}  // namespace

struct ar_ctx {
  std::recursive_mutex mu;   // guards the message and the table caches (a server thread shares them)
  int device = 0;
  int num_sms = 0;
  ar_config cfg{};
  std::string last_error;
  std::vector<PatternDev> patterns;
  std::map<std::pair<int, int>, LenTables> len_tables;                 // (N, k_lo)
  std::map<std::tuple<int, double, int>, int2*> bin_tables;            // (N, fs, pattern)
  std::map<std::pair<int, int>, KernelCfg> unfold_cfg;                 // (N, n_f)
  // per (N, fs): every loaded pattern as the kernels see it (for per-station pattern ids),
  // with the number of patterns it was built for; replaced tables stay allocated until destroy
  std::map<std::pair<int, double>, std::pair<PatternRef*, int>> pattern_refs;
  std::vector<PatternRef*> retired_refs;
  int max_nf = 0;                 // the most frequency nodes of any loaded pattern
  float4* spec = nullptr;
  size_t spec_bytes = 0;
  unsigned* dir_done = nullptr;   // [max directions] completion counters of the fused residual
  DirPre* dir_pre = nullptr;      // [max directions] cells and source vectors, formed per launch
  size_t dir_cap = 0;
  unsigned char* recon = nullptr; // reconstruction state, station times and indices
  size_t recon_bytes = 0;
  unsigned* d_err = nullptr;
  // device staging for ar_unfold_host
  std::vector<std::pair<void*, size_t>> stage;   // slots, grown on demand
  // per-kernel timing
  bool profiling = false;
  int test_fault = 0;        // ar_set_test_fault: 1 makes ar_unfold's corner-slab waits run out
  bool timed = false;
  bool timed_tc = false;   // the last timed call was ar_unfold_tc (four events)
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // tensor-core DFT variant: the split DFT matrices ([0] forward, [1] inverse; 3 BF16 planes
  // each, in the GEMM's shared-memory image) and a workspace for the GEMM operands
  uint4* tc_b[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  unsigned char* tc_ws = nullptr;
  size_t tc_ws_bytes = 0;
};

namespace {

ar_status fail(ar_ctx* ctx, ar_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) {
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    ctx->last_error = buf;
  }
  return st;
}

#define AR_CUDA(ctx, call)                                                                   \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? AR_ERR_OUT_OF_MEMORY : AR_ERR_CUDA, \
                  "%s failed: %s", #call, cudaGetErrorString(e_));                           \
    }                                                                                        \
  } while (0)

// first in-band bin and count; the band is [30, 80] MHz inclusive (same rule as the ABI doc)
void band_window(int n, double fs, int* k_lo, int* count, int* k_hi) {
  *k_lo = -1;
  *count = 0;
  *k_hi = -1;
  for (int k = 0; k < n; ++k) {
    const double f = static_cast<double>(k) * fs / static_cast<double>(n);
    if (f >= kBandLoHz && f <= kBandHiHz) {
      if (*k_lo < 0) *k_lo = k;
      *k_hi = k;
      ++*count;
    }
  }
}

float2 unit(long t, long n, int sign) {   // exp(sign * 2 pi i t / n), t reduced exactly
  t %= n;
  if (t < 0) t += n;
  const double a = 2.0 * M_PI * static_cast<double>(t) / static_cast<double>(n);
  return make_float2(static_cast<float>(std::cos(a)), static_cast<float>(sign * std::sin(a)));
}

// the pass-1 pre-twiddles exp(2 pi i jb r / 4Q) of the 1024- and 4096-sample layouts into the
// kernels' constant tables (current device)
cudaError_t upload_pretwiddles() {
  float2 a[4][32], b[4][16];
  for (int r = 0; r < 4; ++r) {
    for (int j = 0; j < 32; ++j) a[r][j] = unit(static_cast<long>(j) * r, 128, +1);
    for (int j = 0; j < 16; ++j) b[r][j] = unit(static_cast<long>(j) * r, 64, +1);
  }
  cudaError_t e = cudaMemcpyToSymbol(c_pre32, a, sizeof a);
  return e != cudaSuccess ? e : cudaMemcpyToSymbol(c_pre16, b, sizeof b);
}

template <int N_>
ar_status build_len_tables(ar_ctx* ctx, int k_lo, LenTables* lt) {
  using L = Layout<N_>;
  constexpr int N = L::N, Q = L::Q, P = L::P;
  std::vector<float2> t1(4 * Q * P + (L::SPLIT == 1 ? 8 * Q : 0)), wn(N);
  for (int r = 0; r < 4; ++r)
    for (int mb = 0; mb < Q; ++mb)
      for (int ja = 0; ja < P; ++ja)
        t1[(r * Q + mb) * P + ja] = unit(static_cast<long>(k_lo + ja) * (r + 4 * mb), N, +1);
  if (L::SPLIT == 1) {   // pass 2's c = exp(2 pi i P floor(k_lo/P) w / N) and u = exp(2 pi i w / N), w = 4 mb + r
    const long base = static_cast<long>(k_lo / P) * P;
    for (int w = 0; w < 4 * Q; ++w) {
      t1[4 * Q * P + w] = unit(base * w, N, +1);
      t1[4 * Q * P + 4 * Q + w] = unit(w, N, +1);
    }
  }
  for (int t = 0; t < N; ++t) wn[t] = unit(t, N, -1);
  AR_CUDA(ctx, cudaMalloc(&lt->t1, t1.size() * sizeof(float2)));
  AR_CUDA(ctx, cudaMalloc(&lt->wn, wn.size() * sizeof(float2)));
  AR_CUDA(ctx, cudaMemcpy(lt->t1, t1.data(), t1.size() * sizeof(float2), cudaMemcpyHostToDevice));
  AR_CUDA(ctx, cudaMemcpy(lt->wn, wn.data(), wn.size() * sizeof(float2), cudaMemcpyHostToDevice));
  return AR_OK;
}

ar_status get_len_tables(ar_ctx* ctx, int n, int k_lo, LenTables** out) {
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  auto key = std::make_pair(n, k_lo);
  auto it = ctx->len_tables.find(key);
  if (it == ctx->len_tables.end()) {
    LenTables lt;
    ar_status st = n == 1024   ? build_len_tables<1024>(ctx, k_lo, &lt)
                   : n == 2048 ? build_len_tables<2048>(ctx, k_lo, &lt)
                               : build_len_tables<4096>(ctx, k_lo, &lt);
    if (st != AR_OK) return st;
    it = ctx->len_tables.emplace(key, lt).first;
  }
  *out = &it->second;
  return AR_OK;
}

// per window bin: frequency cell of the pattern (or -1 outside the band) and its fraction
ar_status get_bin_table(ar_ctx* ctx, int n, double fs, int pid, int k_lo, int2** out) {
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  auto key = std::make_tuple(n, fs, pid);
  auto it = ctx->bin_tables.find(key);
  if (it == ctx->bin_tables.end()) {
    const ar_pattern_desc& pd = ctx->patterns[pid].desc;
    const int m = n / 4;
    std::vector<int2> bt(m);
    for (int j = 0; j < m; ++j) {
      const int k = k_lo + j;
      const double f = static_cast<double>(k) * fs / static_cast<double>(n);
      if (!(f >= kBandLoHz && f <= kBandHiHz)) {
        bt[j] = make_int2(-1, 0);
        continue;
      }
      double u = (f - pd.f0_hz) / pd.df_hz;
      if (u < 0.0) u = 0.0;
      if (u > static_cast<double>(pd.n_freq - 1)) u = static_cast<double>(pd.n_freq - 1);
      int c = static_cast<int>(std::floor(u));
      if (c > pd.n_freq - 2) c = pd.n_freq - 2;
      const float t = static_cast<float>(u - static_cast<double>(c));
      int tb;
      std::memcpy(&tb, &t, sizeof tb);
      bt[j] = make_int2(c, tb);
    }
    int2* d = nullptr;
    AR_CUDA(ctx, cudaMalloc(&d, bt.size() * sizeof(int2)));
    AR_CUDA(ctx, cudaMemcpy(d, bt.data(), bt.size() * sizeof(int2), cudaMemcpyHostToDevice));
    it = ctx->bin_tables.emplace(key, d).first;
  }
  *out = it->second;
  return AR_OK;
}

// Every loaded pattern at (N, fs) as the kernels see it, indexed by pattern id.
ar_status get_pattern_refs(ar_ctx* ctx, int n, double fs, int k_lo, const PatternRef** out, int* count) {
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  const int np = static_cast<int>(ctx->patterns.size());
  auto key = std::make_pair(n, fs);
  auto it = ctx->pattern_refs.find(key);
  if (it == ctx->pattern_refs.end() || it->second.second != np) {
    std::vector<PatternRef> refs(np);
    for (int i = 0; i < np; ++i) {
      const ar_pattern_desc& pd = ctx->patterns[i].desc;
      int2* binf = nullptr;
      ar_status st = get_bin_table(ctx, n, fs, i, k_lo, &binf);
      if (st != AR_OK) return st;
      refs[i] = PatternRef{ctx->patterns[i].table, binf, pd.zen0_rad, pd.dzen_rad, pd.az0_rad, pd.daz_rad,
                           pd.n_zen, pd.n_az, pd.n_freq, 0};
    }
    PatternRef* d = nullptr;
    AR_CUDA(ctx, cudaMalloc(&d, refs.size() * sizeof(PatternRef)));
    AR_CUDA(ctx, cudaMemcpy(d, refs.data(), refs.size() * sizeof(PatternRef), cudaMemcpyHostToDevice));
    if (it != ctx->pattern_refs.end()) {
      ctx->retired_refs.push_back(it->second.first);   // a launch in flight may still read it
      it->second = {d, np};
    } else {
      it = ctx->pattern_refs.emplace(key, std::make_pair(d, np)).first;
    }
  }
  *out = it->second.first;
  *count = it->second.second;
  return AR_OK;
}

// Per-event workspace of the unfold path: the station band spectra ([S][N/4] float4), then
// (256-byte aligned) the station walk order ([S] int2) used with per-station pattern ids.
size_t walk_offset(int n, long long n_st) {
  return (sizeof(float4) * static_cast<size_t>(n / 4) * static_cast<size_t>(n_st) + 255) / 256 * 256;
}
size_t spec_ws_bytes(int n, long long n_st) { return walk_offset(n, n_st) + sizeof(int2) * static_cast<size_t>(n_st); }

// frequency nodes the unfold kernel lays its shared memory out for
int layout_nf(const ar_ctx* ctx, const ar_event* ev) {
  return ev->station_pattern ? ctx->max_nf : ctx->patterns[ev->pattern_id].desc.n_freq;
}

// per-station patterns: point the descriptor at the pattern table and the caller's ids
ar_status attach_patterns(ar_ctx* ctx, const ar_event* ev, int k_lo, EventDesc* d) {
  if (!ev->station_pattern) return AR_OK;
  const PatternRef* refs = nullptr;
  int count = 0;
  ar_status st = get_pattern_refs(ctx, ev->n_samples, ev->fs_hz, k_lo, &refs, &count);
  if (st != AR_OK) return st;
  d->pats = refs;
  d->st_pat = ev->station_pattern;
  d->st_walk = reinterpret_cast<int2*>(reinterpret_cast<unsigned char*>(d->spec) +
                                       walk_offset(ev->n_samples, ev->n_stations));
  d->n_pats = count;
  d->n_f_layout = ctx->max_nf;
  return AR_OK;
}

ar_status ensure_dirs(ar_ctx* ctx, size_t n_dir) {
  if (n_dir <= ctx->dir_cap) return AR_OK;
  if (ctx->dir_done) {
    AR_CUDA(ctx, cudaDeviceSynchronize());
    AR_CUDA(ctx, cudaFree(ctx->dir_done));
    AR_CUDA(ctx, cudaFree(ctx->dir_pre));
    ctx->dir_done = nullptr;
    ctx->dir_pre = nullptr;
    ctx->dir_cap = 0;
  }
  const size_t cap = std::max<size_t>(n_dir, 256);
  AR_CUDA(ctx, cudaMalloc(&ctx->dir_done, cap * sizeof(unsigned)));
  AR_CUDA(ctx, cudaMemset(ctx->dir_done, 0, cap * sizeof(unsigned)));
  AR_CUDA(ctx, cudaMalloc(&ctx->dir_pre, cap * sizeof(DirPre)));
  ctx->dir_cap = cap;
  return AR_OK;
}

ar_status ensure_spec(ar_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->spec_bytes) return AR_OK;
  if (ctx->spec) {
    AR_CUDA(ctx, cudaDeviceSynchronize());
    AR_CUDA(ctx, cudaFree(ctx->spec));
    ctx->spec = nullptr;
    ctx->spec_bytes = 0;
  }
  AR_CUDA(ctx, cudaMalloc(&ctx->spec, bytes));
  ctx->spec_bytes = bytes;
  return AR_OK;
}

// the dynamic shared-memory limit of both unfold instantiations of a length
template <int N_>
cudaError_t set_unfold_smem_limit(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(unfold_kernel<N_, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(bytes));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(unfold_kernel<N_, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(bytes));
  return e;
}

template <int N_>
ar_status unfold_cfg(ar_ctx* ctx, int n_f, KernelCfg** out) {
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  auto key = std::make_pair(N_, n_f);
  auto it = ctx->unfold_cfg.find(key);
  if (it == ctx->unfold_cfg.end()) {
    KernelCfg kc;
    // the attribute belongs to the kernel, not to this configuration: set it to the largest
    // layout any pattern can need, so that no later set-up lowers it below a cached launch
    AR_CUDA(ctx, set_unfold_smem_limit<N_>(UnfoldSmem<N_>::total(kMaxFreqNodes)));
    // stage the corner slabs by TMA unless that lowers the CTAs per SM (large patterns)
    int per_sm = 0, per_sm_direct = 0;
    AR_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, unfold_kernel<N_, false>, Layout<N_>::T,
                                                               UnfoldSmem<N_>::total(n_f)));
    AR_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_direct, unfold_kernel<N_, false>, Layout<N_>::T,
                                                               UnfoldSmem<N_>::total(n_f, true)));
    kc.slab_direct = per_sm_direct > per_sm ? 1 : 0;
    if (kc.slab_direct) per_sm = per_sm_direct;
    kc.smem = UnfoldSmem<N_>::total(n_f, kc.slab_direct != 0);
    if (per_sm < 1) return fail(ctx, AR_ERR_CUDA, "unfold kernel N=%d does not fit an SM (smem %zu)", N_, kc.smem);
    kc.grid = per_sm * ctx->num_sms;
    AR_CUDA(ctx, cudaFuncSetAttribute(station_spectrum_kernel<N_>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(SpectrumSmem<N_>::TOTAL)));
    it = ctx->unfold_cfg.emplace(key, kc).first;
  }
  *out = &it->second;
  return AR_OK;
}

struct Resolved {
  int k_lo = 0;
  LenTables* lt = nullptr;
  int2* binf = nullptr;
  KernelCfg* kc = nullptr;
};

ar_status validate_shape(ar_ctx* ctx, int n, double fs, int pid, int* k_lo) {
  if (n != 1024 && n != 2048 && n != 4096)
    return fail(ctx, AR_ERR_UNSUPPORTED_N, "n_samples=%d: supported lengths are 1024, 2048, 4096", n);
  if (!(fs > 0.0) || !std::isfinite(fs)) return fail(ctx, AR_ERR_INVALID_ARG, "fs_hz=%g must be positive", fs);
  if (pid < 0 || pid >= static_cast<int>(ctx->patterns.size()))
    return fail(ctx, AR_ERR_NO_PATTERN, "pattern_id=%d was not loaded", pid);
  int lo, cnt, hi;
  band_window(n, fs, &lo, &cnt, &hi);
  if (cnt < 1) return fail(ctx, AR_ERR_INVALID_ARG, "no bin of N=%d at fs=%g Hz lies in 30-80 MHz", n, fs);
  if (cnt > n / 4 || lo + n / 4 > n / 2 || 2 * hi >= n)
    return fail(ctx, AR_ERR_INVALID_ARG,
                "fs=%g Hz: the 30-80 MHz band (%d bins from %d) must fit N/4 bins below Nyquist", fs, cnt, lo);
  *k_lo = lo;
  return AR_OK;
}

ar_status resolve(ar_ctx* ctx, int n, double fs, int pid, int max_st, Resolved* rs, int n_f_layout = 0) {
  ar_status st = validate_shape(ctx, n, fs, pid, &rs->k_lo);
  if (st != AR_OK) return st;
  if ((st = get_len_tables(ctx, n, rs->k_lo, &rs->lt)) != AR_OK) return st;
  if ((st = get_bin_table(ctx, n, fs, pid, rs->k_lo, &rs->binf)) != AR_OK) return st;
  const int n_f = n_f_layout > 0 ? n_f_layout : ctx->patterns[pid].desc.n_freq;
  st = n == 1024 ? unfold_cfg<1024>(ctx, n_f, &rs->kc)
       : n == 2048 ? unfold_cfg<2048>(ctx, n_f, &rs->kc)
                   : unfold_cfg<4096>(ctx, n_f, &rs->kc);
  if (st != AR_OK) return st;
  return ensure_spec(ctx, spec_ws_bytes(n, max_st));
}

ar_status resolve_dirs(ar_ctx* ctx, int n_dir) { return ensure_dirs(ctx, static_cast<size_t>(n_dir)); }

// Launch with programmatic dependent launch allowed: the kernel may start while the previous
// kernel in the stream finishes; it waits (griddepcontrol.wait) before touching its results.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t stream,
                       Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

struct PathBuffers {      // library-side buffers one launch of the path uses
  float4* spec;
  unsigned* dir_done;
  unsigned* err;
  const float2* t1;
  const float2* wn;
  const int2* binf;
  DirPre* dir_pre = nullptr;   // [D] per-direction precomputation by the station kernel, or none
};

// the kernels' view of one event (see EventDesc)
EventDesc make_desc(const PathBuffers& b, const ar_pattern_desc& pd, const float2* table, const ar_event* ev,
                    const ar_outputs* out, int k_lo) {
  EventDesc d{};
  d.traces = ev->traces;
  d.pos = ev->pos_m;
  d.t_start = ev->t_start_ns;
  d.dirs = ev->dirs_rad;
  d.efield = out->efield;
  d.envelope = out->envelope;
  d.peak_idx = out->peak_idx;
  d.peak_amp = out->peak_amp;
  d.peak_time = out->peak_time_ns;
  d.peak_fine = out->peak_time_fine_ns;
  d.snr = out->snr;
  d.status = out->status;
  d.residual = out->residual_ns;
  d.t0 = out->t0_ns;
  d.chi2 = out->chi2;
  d.spec = b.spec;
  d.dir_done = b.dir_done;
  d.dir_pre = b.dir_pre;
  d.table = table;
  d.binf = b.binf;
  d.t1 = b.t1;
  d.wn = b.wn;
  d.zen0 = pd.zen0_rad;
  d.dzen = pd.dzen_rad;
  d.az0 = pd.az0_rad;
  d.daz = pd.daz_rad;
  d.dt_ns = 1e9 / ev->fs_hz;
  d.n_over_c = (ev->refractive_index > 0.0 ? ev->refractive_index : 1.0) / kCMPerNs;
  d.inv_n_st = 1.0 / static_cast<double>(ev->n_stations);
  d.pair_begin = 0;
  d.station_begin = 0;
  d.n_zen = pd.n_zen;
  d.n_az = pd.n_az;
  d.n_f = pd.n_freq;
  d.n_f_layout = pd.n_freq;
  d.n_st = ev->n_stations;
  d.n_dir = ev->n_dirs;
  d.k_lo = k_lo;
  return d;
}

// One event: the station kernel (one CTA per station), then the persistent unfold kernel.
// The station kernel is launched in plain stream order: launched early behind the previous
// call's unfold kernel it would hold SM slots that kernel's successor needs (back to back,
// calls took 0.124 instead of 0.095 ms on the scan). The unfold kernel is launched with
// programmatic dependent launch, so its CTAs start while the station kernel runs and fetch
// their first corner slabs before they wait for the spectra.
template <int N_>
cudaError_t launch_path(unsigned* err, const EventDesc& desc, int grid_cap, cudaStream_t stream,
                        cudaEvent_t* evs /* 3 events or null */, int test_wait = 0) {
  using L = Layout<N_>;
  PathParams pp{};
  pp.batch = nullptr;
  pp.err = err;
  pp.wait_prior = 1;
  pp.test_wait = test_wait;
  pp.ev0 = desc;
  cudaError_t e;
  if (evs && (e = cudaEventRecord(evs[0], stream)) != cudaSuccess) return e;
  station_spectrum_kernel<N_><<<desc.n_st, SpectrumSmem<N_>::BLOCK, SpectrumSmem<N_>::TOTAL, stream>>>(pp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (evs && (e = cudaEventRecord(evs[1], stream)) != cudaSuccess) return e;
  const long long pairs = static_cast<long long>(desc.n_st) * desc.n_dir;
  const long long grid = std::min<long long>(grid_cap, pairs);
  const size_t smem = UnfoldSmem<N_>::total(pp.ev0.n_f_layout, pp.ev0.slab_direct != 0);
  if ((e = desc.snr ? launch_pdl(unfold_kernel<N_, true>, static_cast<int>(grid), L::T, smem, stream, pp)
                    : launch_pdl(unfold_kernel<N_, false>, static_cast<int>(grid), L::T, smem, stream, pp)) !=
      cudaSuccess)
    return e;
  if (evs && (e = cudaEventRecord(evs[2], stream)) != cudaSuccess) return e;
  return cudaSuccess;
}

template <int N_>
ar_status launch_all(ar_ctx* ctx, const ar_event* ev, const ar_outputs* out, const Resolved& rs,
                     cudaStream_t stream) {
  const PatternDev& pat = ctx->patterns[ev->pattern_id];
  PathBuffers b{ctx->spec, ctx->dir_done, ctx->d_err, rs.lt->t1, rs.lt->wn, rs.binf, ctx->dir_pre};
  EventDesc desc = make_desc(b, pat.desc, pat.table, ev, out, rs.k_lo);
  ar_status st = attach_patterns(ctx, ev, rs.k_lo, &desc);
  if (st != AR_OK) return st;
  desc.slab_direct = rs.kc->slab_direct;
  cudaError_t e = launch_path<N_>(ctx->d_err, desc, rs.kc->grid, stream, ctx->profiling ? ctx->ev : nullptr,
                                  ctx->test_fault);
  if (e != cudaSuccess) return fail(ctx, AR_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
  if (ctx->profiling) {
    ctx->timed = true;
    ctx->timed_tc = false;
  }
  return AR_OK;
}

// The checks of a pattern descriptor that ar_load_pattern and ar_unfold_noalloc share: false
// if it is valid, else true with the reason in why.
bool pattern_desc_error(const ar_pattern_desc* d, char* why, size_t n) {
  if (d->n_zen < 2 || d->n_az < 2 || d->n_freq < 2 || d->n_freq > kMaxFreqNodes) {
    snprintf(why, n, "pattern sizes %d x %d x %d out of range", d->n_zen, d->n_az, d->n_freq);
    return true;
  }
  if (!(d->dzen_rad > 0) || !(d->daz_rad > 0) || !(d->df_hz > 0) || !std::isfinite(d->dzen_rad) ||
      !std::isfinite(d->daz_rad) || !std::isfinite(d->df_hz) || !std::isfinite(d->zen0_rad) ||
      !std::isfinite(d->az0_rad) || !std::isfinite(d->f0_hz)) {
    snprintf(why, n, "pattern axis steps must be positive and finite, origins finite");
    return true;
  }
  if (std::fabs(d->n_az * d->daz_rad - 2.0 * M_PI) > 1e-9 * 2.0 * M_PI) {
    snprintf(why, n, "azimuth axis must cover 2 pi (n_az * daz = %.17g)", d->n_az * d->daz_rad);
    return true;
  }
  const size_t nodes = static_cast<size_t>(d->n_zen) * d->n_az * d->n_freq;
  if (nodes * 4 > (1ull << 31)) {
    snprintf(why, n, "pattern too large (%zu nodes)", nodes);
    return true;
  }
  return false;
}

// The checks of an event and its outputs that every entry point shares (the trace length and
// rate are checked with the band window): false if they pass, else true with the reason.
bool event_error(const ar_event* ev, const ar_outputs* out, char* why, size_t n) {
  if (!ev || !out) return snprintf(why, n, "event and outputs must not be NULL"), true;
  if (ev->n_stations < 1 || ev->n_stations > (1 << 20))
    return snprintf(why, n, "n_stations=%d out of [1, 2^20]", ev->n_stations), true;
  if (ev->n_dirs < 1 || ev->n_dirs > (1 << 20)) return snprintf(why, n, "n_dirs=%d out of [1, 2^20]", ev->n_dirs), true;
  if (!ev->traces || !ev->pos_m || !ev->t_start_ns || !ev->dirs_rad)
    return snprintf(why, n, "event arrays must not be NULL"), true;
  if (reinterpret_cast<uintptr_t>(ev->traces) % 16 != 0) return snprintf(why, n, "traces must be 16-byte aligned"), true;
  if (!out->peak_idx || !out->peak_amp || !out->peak_time_ns || !out->residual_ns || !out->t0_ns || !out->chi2 ||
      !out->status)
    return snprintf(why, n, "peak, residual and status outputs must not be NULL"), true;
  if (!(ev->refractive_index >= 0.0) || !std::isfinite(ev->refractive_index))
    return snprintf(why, n, "refractive_index must be finite and >= 0"), true;
  if (reinterpret_cast<uintptr_t>(out->efield) % 16 != 0 || reinterpret_cast<uintptr_t>(out->envelope) % 16 != 0)
    return snprintf(why, n, "efield and envelope must be 16-byte aligned"), true;
  if (!out->efield && out->envelope)
    return snprintf(why, n, "envelope without efield is not supported (give both or neither)"), true;
  return false;
}

ar_status check_event(ar_ctx* ctx, const ar_event* ev, const ar_outputs* out) {
  char why[256];
  if (event_error(ev, out, why, sizeof why)) return fail(ctx, AR_ERR_INVALID_ARG, "%s", why);
  return AR_OK;
}

}  // namespace

extern "C" {

const char* ar_status_string(ar_status s) {
  switch (s) {
    case AR_OK: return "AR_OK";
    case AR_ERR_INVALID_ARG: return "AR_ERR_INVALID_ARG";
    case AR_ERR_UNSUPPORTED_N: return "AR_ERR_UNSUPPORTED_N";
    case AR_ERR_NO_PATTERN: return "AR_ERR_NO_PATTERN";
    case AR_ERR_OUT_OF_MEMORY: return "AR_ERR_OUT_OF_MEMORY";
    case AR_ERR_BUDGET: return "AR_ERR_BUDGET";
    case AR_ERR_CUDA: return "AR_ERR_CUDA";
    case AR_ERR_TIMEOUT: return "AR_ERR_TIMEOUT";
    case AR_ERR_NOT_READY: return "AR_ERR_NOT_READY";
    case AR_ERR_DEVICE: return "AR_ERR_DEVICE";
  }
  return "AR_ERR_UNKNOWN";
}

ar_status ar_create(ar_ctx** out, const ar_config* cfg) {
  if (!out) return AR_ERR_INVALID_ARG;
  *out = nullptr;
  ar_config c{};
  if (cfg) c = *cfg;
  if (c.state_budget_bytes == 0) c.state_budget_bytes = 4ull << 30;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  auto create_fail = [&](ar_status st, const char* msg) {
    g_create_error = msg;
    return st;
  };
  if (e != cudaSuccess) return create_fail(AR_ERR_CUDA, cudaGetErrorString(e));
  if (c.device < 0 || c.device >= ndev) return create_fail(AR_ERR_CUDA, "no such CUDA device");
  if ((e = cudaSetDevice(c.device)) != cudaSuccess) return create_fail(AR_ERR_CUDA, cudaGetErrorString(e));
  ar_ctx* ctx = new ar_ctx;
  ctx->device = c.device;
  ctx->cfg = c;
  if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess ||
      cudaMalloc(&ctx->d_err, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(ctx->d_err, 0, sizeof(unsigned)) != cudaSuccess || upload_pretwiddles() != cudaSuccess) {
    delete ctx;
    return create_fail(AR_ERR_OUT_OF_MEMORY, "context allocation failed");
  }
  *out = ctx;
  return AR_OK;
}

ar_status ar_destroy(ar_ctx* ctx) {
  if (!ctx) return AR_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto& p : ctx->patterns) cudaFree(p.table);
  for (auto& kv : ctx->len_tables) {
    cudaFree(kv.second.t1);
    cudaFree(kv.second.wn);
  }
  for (auto& kv : ctx->bin_tables) cudaFree(kv.second);
  for (auto& kv : ctx->pattern_refs) cudaFree(kv.second.first);
  for (auto* p : ctx->retired_refs) cudaFree(p);
  for (auto& s : ctx->stage) cudaFree(s.first);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  cudaFree(ctx->spec);
  cudaFree(ctx->dir_done);
  cudaFree(ctx->dir_pre);
  cudaFree(ctx->recon);
  for (auto& m : ctx->tc_b)
    for (auto* p : m) cudaFree(p);
  cudaFree(ctx->tc_ws);
  cudaFree(ctx->d_err);
  delete ctx;
  return AR_OK;
}

const char* ar_last_error(const ar_ctx* ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->last_error.c_str();
}

ar_status ar_load_pattern(ar_ctx* ctx, const ar_pattern_desc* d, const float* host_table, int32_t* pattern_id) {
  if (!ctx) return AR_ERR_INVALID_ARG;
  if (!d || !host_table || !pattern_id) return fail(ctx, AR_ERR_INVALID_ARG, "NULL argument");
  char why[256];
  if (pattern_desc_error(d, why, sizeof why)) return fail(ctx, AR_ERR_INVALID_ARG, "%s", why);
  const size_t nodes = static_cast<size_t>(d->n_zen) * d->n_az * d->n_freq;
  AR_CUDA(ctx, cudaSetDevice(ctx->device));
  PatternDev p;
  p.desc = *d;
  p.bytes = nodes * 4 * sizeof(float2);
  AR_CUDA(ctx, cudaMalloc(&p.table, p.bytes));
  cudaError_t e = cudaMemcpy(p.table, host_table, p.bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(p.table);
    return fail(ctx, AR_ERR_CUDA, "pattern upload failed: %s", cudaGetErrorString(e));
  }
  ctx->patterns.push_back(p);
  ctx->max_nf = std::max(ctx->max_nf, d->n_freq);
  *pattern_id = static_cast<int32_t>(ctx->patterns.size() - 1);
  return AR_OK;
}

ar_status ar_prepare(ar_ctx* ctx, int32_t n_samples, double fs_hz, int32_t pattern_id, int32_t max_stations) {
  if (!ctx) return AR_ERR_INVALID_ARG;
  if (max_stations < 1) return fail(ctx, AR_ERR_INVALID_ARG, "max_stations must be >= 1");
  AR_CUDA(ctx, cudaSetDevice(ctx->device));
  Resolved rs;
  return resolve(ctx, n_samples, fs_hz, pattern_id, max_stations, &rs);
}

ar_status ar_unfold(ar_ctx* ctx, const ar_event* ev, const ar_outputs* out, void* stream) {
  NvtxRange nvtx("ar_unfold");
  if (!ctx) return AR_ERR_INVALID_ARG;
  ar_status st = check_event(ctx, ev, out);
  if (st != AR_OK) return st;
  AR_CUDA(ctx, cudaSetDevice(ctx->device));
  Resolved rs;
  if ((st = resolve(ctx, ev->n_samples, ev->fs_hz, ev->pattern_id, ev->n_stations, &rs, layout_nf(ctx, ev))) !=
      AR_OK)
    return st;
  if ((st = resolve_dirs(ctx, ev->n_dirs)) != AR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (ev->n_samples) {
    case 1024: return launch_all<1024>(ctx, ev, out, rs, s);
    case 2048: return launch_all<2048>(ctx, ev, out, rs, s);
    default: return launch_all<4096>(ctx, ev, out, rs, s);
  }
}

}  // extern "C"

namespace {

template <int N_>
cudaError_t launch_recon(ar_ctx* ctx, const ar_event* ev, int max_iter, double tol_rad, const ar_recon_out* out,
                         const Resolved& rs, ReconState* st, int* vidx, double* vtimes, int* prev_idx,
                         cudaStream_t stream) {
  using L = Layout<N_>;
  const PatternDev& pat = ctx->patterns[ev->pattern_id];
  ar_event e1 = *ev;
  e1.n_dirs = 1;
  e1.dirs_rad = st->dir;   // the direction the last fit produced (device memory)
  PathBuffers b{ctx->spec, ctx->dir_done, ctx->d_err, rs.lt->t1, rs.lt->wn, rs.binf};
  PathParams pp{};
  pp.batch = nullptr;
  pp.err = ctx->d_err;
  pp.skip = &st->converged;
  pp.wait_prior = 1;
  pp.ev0 = make_desc(b, pat.desc, pat.table, &e1, &out->last, rs.k_lo);
  if (attach_patterns(ctx, &e1, rs.k_lo, &pp.ev0) != AR_OK) return cudaErrorMemoryAllocation;
  pp.ev0.slab_direct = rs.kc->slab_direct;
  const int S = ev->n_stations;
  const double dt_ns = 1e9 / ev->fs_hz;
  const double n_over_c = (ev->refractive_index > 0.0 ? ev->refractive_index : 1.0) / kCMPerNs;
  cudaError_t e = cudaMemsetAsync(st, 0, sizeof(ReconState), stream);
  if (e == cudaSuccess && out->history)
    e = cudaMemsetAsync(out->history, 0xff, sizeof(double) * 2 * (max_iter + 1), stream);   // NaN
  if (e != cudaSuccess) return e;
  // the station spectra, once: every iteration unfolds the same traces
  PathParams sp = pp;
  sp.skip = nullptr;
  station_spectrum_kernel<N_><<<S, SpectrumSmem<N_>::BLOCK, SpectrumSmem<N_>::TOTAL, stream>>>(sp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  voltage_peak_kernel<<<S, 256, 0, stream>>>(ev->traces, ev->t_start_ns, ev->n_samples, dt_ns, vidx, vtimes);
  FitParams fp{ev->pos_m, vtimes, vidx, prev_idx, st, out->history, n_over_c, tol_rad, S, 0};
  plane_fit_kernel<<<1, 128, 0, stream>>>(fp);
  for (int it = 1; it <= max_iter; ++it) {
    const size_t smem = UnfoldSmem<N_>::total(pp.ev0.n_f_layout, pp.ev0.slab_direct != 0);
    if ((e = pp.ev0.snr ? launch_pdl(unfold_kernel<N_, true>, std::min(rs.kc->grid, S), L::T, smem, stream, pp)
                        : launch_pdl(unfold_kernel<N_, false>, std::min(rs.kc->grid, S), L::T, smem, stream, pp)) !=
        cudaSuccess)
      return e;
    fp.times = out->last.peak_time_ns;
    fp.idx = out->last.peak_idx;
    fp.iteration = it;
    plane_fit_kernel<<<1, 128, 0, stream>>>(fp);
  }
  recon_finish_kernel<<<1, 32, 0, stream>>>(st, out->direction, out->t0_ns, out->chi2, out->iterations);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

ar_status ar_reconstruct(ar_ctx* ctx, const ar_event* ev, int32_t max_iter, double tol_rad, const ar_recon_out* out,
                         void* stream) {
  NvtxRange nvtx("ar_reconstruct");
  if (!ctx) return AR_ERR_INVALID_ARG;
  if (!ev || !out) return fail(ctx, AR_ERR_INVALID_ARG, "event and outputs must not be NULL");
  if (max_iter < 0 || max_iter > 64) return fail(ctx, AR_ERR_INVALID_ARG, "max_iter must be in [0, 64]");
  if (!(tol_rad >= 0.0)) return fail(ctx, AR_ERR_INVALID_ARG, "tol_rad must be >= 0");
  if (!out->direction || !out->t0_ns || !out->chi2 || !out->iterations)
    return fail(ctx, AR_ERR_INVALID_ARG, "direction, t0, chi2 and iterations outputs must not be NULL");
  ar_event e1 = *ev;
  e1.n_dirs = 1;
  e1.dirs_rad = reinterpret_cast<const double*>(ev->traces);   // placeholder for validation only
  ar_status st = check_event(ctx, &e1, &out->last);
  if (st != AR_OK) return st;
  if (ev->n_stations < 3) return fail(ctx, AR_ERR_INVALID_ARG, "a direction fit needs at least 3 stations");
  AR_CUDA(ctx, cudaSetDevice(ctx->device));
  Resolved rs;
  if ((st = resolve(ctx, ev->n_samples, ev->fs_hz, ev->pattern_id, ev->n_stations, &rs, layout_nf(ctx, ev))) !=
      AR_OK)
    return st;
  if ((st = resolve_dirs(ctx, 1)) != AR_OK) return st;
  {
    EventDesc probe{};
    if ((st = attach_patterns(ctx, ev, rs.k_lo, &probe)) != AR_OK) return st;   // builds the pattern table
  }
  const size_t S = ev->n_stations;
  const size_t need = 256 + S * (4 + 8 + 4) + 3 * 256;
  if (need > ctx->recon_bytes) {
    AR_CUDA(ctx, cudaDeviceSynchronize());
    cudaFree(ctx->recon);
    ctx->recon = nullptr;
    ctx->recon_bytes = 0;
    AR_CUDA(ctx, cudaMalloc(&ctx->recon, need));
    ctx->recon_bytes = need;
  }
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  ReconState* rst = reinterpret_cast<ReconState*>(ctx->recon);
  double* vtimes = reinterpret_cast<double*>(ctx->recon + 256);
  int* vidx = reinterpret_cast<int*>(ctx->recon + 256 + up(S * 8));
  int* prev_idx = reinterpret_cast<int*>(ctx->recon + 256 + up(S * 8) + up(S * 4));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = ev->n_samples == 1024 ? launch_recon<1024>(ctx, ev, max_iter, tol_rad, out, rs, rst, vidx, vtimes, prev_idx, s)
                  : ev->n_samples == 2048 ? launch_recon<2048>(ctx, ev, max_iter, tol_rad, out, rs, rst, vidx, vtimes, prev_idx, s)
                                          : launch_recon<4096>(ctx, ev, max_iter, tol_rad, out, rs, rst, vidx, vtimes, prev_idx, s);
  if (e != cudaSuccess) return fail(ctx, AR_ERR_CUDA, "reconstruction launch failed: %s", cudaGetErrorString(e));
  return AR_OK;
}

ar_status ar_sync(ar_ctx* ctx, void* stream) {
  if (!ctx) return AR_ERR_INVALID_ARG;
  AR_CUDA(ctx, cudaSetDevice(ctx->device));
  AR_CUDA(ctx, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  unsigned err = 0;
  AR_CUDA(ctx, cudaMemcpy(&err, ctx->d_err, sizeof err, cudaMemcpyDeviceToHost));
  if (err) {
    AR_CUDA(ctx, cudaMemset(ctx->d_err, 0, sizeof(unsigned)));
    return fail(ctx, AR_ERR_DEVICE,
                "device error 0x%x (bit 0: a bounded wait for a bulk copy ran out; bit 1: a kernel got a launch "
                "configuration it does not take; bit 2: an index check of the debug build failed)",
                err);
  }
  return AR_OK;
}

ar_status ar_unfold_host(ar_ctx* ctx, const ar_event* ev, const ar_outputs* out, void* stream) {
  NvtxRange nvtx("ar_unfold_host");
  if (!ctx) return AR_ERR_INVALID_ARG;
  ar_status st = check_event(ctx, ev, out);
  if (st != AR_OK) return st;
  AR_CUDA(ctx, cudaSetDevice(ctx->device));
  const size_t S = ev->n_stations, D = ev->n_dirs, N = ev->n_samples;
  if (N != 1024 && N != 2048 && N != 4096)
    return fail(ctx, AR_ERR_UNSUPPORTED_N, "n_samples=%zu: supported lengths are 1024, 2048, 4096", N);
  // staging slots: 0 traces, 1 pos, 2 t_start, 3 dirs, 4 efield, 5 envelope, 6 peak_idx,
  // 7 peak_amp, 8 peak_time, 9 residual, 10 t0, 11 chi2, 12 status, 13 station patterns,
  // 14 fine peak times, 15 SNRs
  const size_t sizes[16] = {S * 2 * N * sizeof(float), S * 3 * sizeof(double), S * sizeof(double),
                            D * 2 * sizeof(double), out->efield ? D * S * 2 * N * sizeof(float) : 0,
                            out->envelope ? D * S * N * sizeof(float) : 0, D * S * sizeof(int32_t),
                            D * S * sizeof(float), D * S * sizeof(double), D * S * sizeof(double),
                            D * sizeof(double), D * sizeof(double), D * S * sizeof(uint32_t),
                            ev->station_pattern ? S * sizeof(int32_t) : 0,
                            out->peak_time_fine_ns ? D * S * sizeof(double) : 0,
                            out->snr ? D * S * sizeof(float) : 0};
  if (ctx->stage.size() < 16) ctx->stage.resize(16, {nullptr, 0});
  for (int i = 0; i < 16; ++i) {
    if (sizes[i] > ctx->stage[i].second) {
      AR_CUDA(ctx, cudaDeviceSynchronize());
      cudaFree(ctx->stage[i].first);
      ctx->stage[i] = {nullptr, 0};
      AR_CUDA(ctx, cudaMalloc(&ctx->stage[i].first, sizes[i]));
      ctx->stage[i].second = sizes[i];
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto dev = [&](int i) { return ctx->stage[i].first; };
  AR_CUDA(ctx, cudaMemcpyAsync(dev(0), ev->traces, sizes[0], cudaMemcpyHostToDevice, s));
  AR_CUDA(ctx, cudaMemcpyAsync(dev(1), ev->pos_m, sizes[1], cudaMemcpyHostToDevice, s));
  AR_CUDA(ctx, cudaMemcpyAsync(dev(2), ev->t_start_ns, sizes[2], cudaMemcpyHostToDevice, s));
  AR_CUDA(ctx, cudaMemcpyAsync(dev(3), ev->dirs_rad, sizes[3], cudaMemcpyHostToDevice, s));
  if (ev->station_pattern)
    AR_CUDA(ctx, cudaMemcpyAsync(dev(13), ev->station_pattern, sizes[13], cudaMemcpyHostToDevice, s));
  ar_event de = *ev;
  de.station_pattern = ev->station_pattern ? static_cast<const int32_t*>(dev(13)) : nullptr;
  de.traces = static_cast<const float*>(dev(0));
  de.pos_m = static_cast<const double*>(dev(1));
  de.t_start_ns = static_cast<const double*>(dev(2));
  de.dirs_rad = static_cast<const double*>(dev(3));
  ar_outputs dout{};
  dout.efield = out->efield ? static_cast<float*>(dev(4)) : nullptr;
  dout.envelope = out->envelope ? static_cast<float*>(dev(5)) : nullptr;
  dout.peak_idx = static_cast<int32_t*>(dev(6));
  dout.peak_amp = static_cast<float*>(dev(7));
  dout.peak_time_ns = static_cast<double*>(dev(8));
  dout.residual_ns = static_cast<double*>(dev(9));
  dout.t0_ns = static_cast<double*>(dev(10));
  dout.chi2 = static_cast<double*>(dev(11));
  dout.status = static_cast<uint32_t*>(dev(12));
  dout.peak_time_fine_ns = out->peak_time_fine_ns ? static_cast<double*>(dev(14)) : nullptr;
  dout.snr = out->snr ? static_cast<float*>(dev(15)) : nullptr;
  if ((st = ar_unfold(ctx, &de, &dout, stream)) != AR_OK) return st;
  void* hosts[16] = {nullptr, nullptr, nullptr, nullptr, out->efield, out->envelope, out->peak_idx,
                     out->peak_amp, out->peak_time_ns, out->residual_ns, out->t0_ns, out->chi2, out->status,
                     nullptr, out->peak_time_fine_ns, out->snr};
  for (int i = 4; i < 16; ++i)
    if (hosts[i] && sizes[i]) AR_CUDA(ctx, cudaMemcpyAsync(hosts[i], dev(i), sizes[i], cudaMemcpyDeviceToHost, s));
  return ar_sync(ctx, stream);
}

ar_status ar_set_test_fault(ar_ctx* ctx, int32_t mode) {
  if (!ctx) return AR_ERR_INVALID_ARG;
  if (mode != 0 && mode != 1) return fail(ctx, AR_ERR_INVALID_ARG, "test fault mode %d: 0 or 1", mode);
  ctx->test_fault = mode;
  return AR_OK;
}

ar_status ar_set_profiling(ar_ctx* ctx, int32_t enable) {
  if (!ctx) return AR_ERR_INVALID_ARG;
  AR_CUDA(ctx, cudaSetDevice(ctx->device));
  if (enable && !ctx->ev[0])
    for (auto& e : ctx->ev) AR_CUDA(ctx, cudaEventCreate(&e));
  ctx->profiling = enable != 0;
  ctx->timed = false;
  return AR_OK;
}

ar_status ar_kernel_times(ar_ctx* ctx, float* ms) {
  if (!ctx) return AR_ERR_INVALID_ARG;
  if (!ms || !ctx->timed) return fail(ctx, AR_ERR_INVALID_ARG, "no timed ar_unfold to report");
  AR_CUDA(ctx, cudaEventSynchronize(ctx->ev[2]));
  if (ctx->timed_tc) {
    AR_CUDA(ctx, cudaEventSynchronize(ctx->ev[3]));
    AR_CUDA(ctx, cudaEventElapsedTime(&ms[0], ctx->ev[0], ctx->ev[1]));
    AR_CUDA(ctx, cudaEventElapsedTime(&ms[1], ctx->ev[1], ctx->ev[2]));
    AR_CUDA(ctx, cudaEventElapsedTime(&ms[2], ctx->ev[2], ctx->ev[3]));
    return AR_OK;
  }
  AR_CUDA(ctx, cudaEventElapsedTime(&ms[0], ctx->ev[0], ctx->ev[1]));
  AR_CUDA(ctx, cudaEventElapsedTime(&ms[1], ctx->ev[1], ctx->ev[2]));
  ms[2] = 0.0f;   // the residual runs inside the unfold kernel
  return AR_OK;
}

}  // extern "C"

// ---- tensor-core DFT variant --------------------------------------------------------------
//
// The forward and inverse transforms as split-BF16 GEMMs on tcgen05 tensor cores (tc_dft.cuh):
// per call, the pre-pass and the forward GEMM over all stations, then per chunk of pairs the
// solve, the inverse GEMM and the post-pass, then the per-direction residual.

namespace {

constexpr long long kTcMaxStationSamples = 1ll << 24;   // S * N: bounds the forward workspace
constexpr long long kTcChunkSamples = 1ll << 25;        // pairs * N per inverse chunk

// round to the nearest BF16 (8 significant bits, ties to even) from FP64, as BF16 bits
uint16_t bf16_bits(double x, double* value) {
  if (x == 0.0) {
    *value = 0.0;
    return 0;
  }
  int e = 0;
  std::frexp(x, &e);   // |x| = m 2^e, 0.5 <= m < 1
  const double q = std::ldexp(std::nearbyint(std::ldexp(x, 8 - e)), e - 8);
  *value = q;
  const float f = static_cast<float>(q);   // exact: 8 significant bits
  uint32_t u;
  std::memcpy(&u, &f, sizeof u);
  return static_cast<uint16_t>(u >> 16);
}

// The two real DFT matrices of the four-step transforms, split into three BF16 planes from
// FP64 and laid out as the GEMM's shared-memory image. Rows are output columns, columns the
// K index; complex values are interleaved (re, im).
//   forward  (256 x 1024): X[j2] = sum_n2 W[n2] e^{-2 pi i j2 n2/512}
//   inverse (1024 x 256):  Y[n2] = sum_j2 Z[j2] e^{+2 pi i j2 n2/512}
ar_status build_tc_tables(ar_ctx* ctx) {
  if (ctx->tc_b[0][0]) return AR_OK;
  for (int which = 0; which < 2; ++which) {
    const int rows = which == 0 ? tc::kFwdN : tc::kInvN;
    const int cols = which == 0 ? tc::kFwdK : tc::kInvK;
    std::vector<uint16_t> img[3];
    for (auto& v : img) v.assign(static_cast<size_t>(rows) * cols, 0);
    for (int r = 0; r < rows; ++r) {
      for (int c = 0; c < cols; ++c) {
        const int out_bin = r >> 1, out_part = r & 1, in_bin = c >> 1, in_part = c & 1;
        const long t = (static_cast<long>(out_bin) * in_bin) % tc::kSub;
        const double a = 2.0 * M_PI * static_cast<double>(t) / tc::kSub;
        const double cs = std::cos(a), sn = which == 0 ? -std::sin(a) : std::sin(a);
        // (re, im) of the output from (re, im) of the input: [[cs, -sn], [sn, cs]]
        const double v = out_part == 0 ? (in_part == 0 ? cs : -sn) : (in_part == 0 ? sn : cs);
        double h, m, l;
        const uint16_t bh = bf16_bits(v, &h);
        const uint16_t bm = bf16_bits(v - h, &m);
        const uint16_t bl = bf16_bits(v - h - m, &l);
        const size_t idx = tc::image_offset(r, c, cols);
        img[0][idx] = bh;
        img[1][idx] = bm;
        img[2][idx] = bl;
      }
    }
    for (int pl = 0; pl < 3; ++pl) {
      const size_t bytes = img[pl].size() * sizeof(uint16_t);
      AR_CUDA(ctx, cudaMalloc(&ctx->tc_b[which][pl], bytes));
      AR_CUDA(ctx, cudaMemcpy(ctx->tc_b[which][pl], img[pl].data(), bytes, cudaMemcpyHostToDevice));
    }
  }
  AR_CUDA(ctx, cudaFuncSetAttribute(tc::split_gemm_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(tc::kGemmSmem)));
  AR_CUDA(ctx, cudaFuncSetAttribute(tc::split_gemm_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(tc::kGemmSmem)));
  return AR_OK;
}

size_t pad128(size_t x) { return (x + 127) / 128 * 128; }
size_t pad256b(size_t bytes) { return (bytes + 255) / 256 * 256; }

// Workspace of one call: the two GEMMs' A images (BF16, up to 3 planes), their FP32 outputs,
// and the split-K partial results.
struct TcWorkspace {
  __nv_bfloat16* fa[3];   // forward A image: rows_f x 1024
  float* xf;              // forward D: rows_f x 256
  __nv_bfloat16* za[3];   // inverse A image: rows_c x 256
  float* yi;              // inverse D: rows_c x 1024
  float* part;            // split-K partials: 2 x 128 x 128 floats per CTA of the grid
  size_t bytes;
};

TcWorkspace tc_layout(unsigned char* base, size_t rows_f, size_t rows_c, int num_sms) {
  TcWorkspace w{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base ? base + off : nullptr;
    off += pad256b(bytes);
    return p;
  };
  for (auto& x : w.fa) x = reinterpret_cast<__nv_bfloat16*>(take(rows_f * tc::kFwdK * 2));
  w.xf = reinterpret_cast<float*>(take(rows_f * tc::kFwdN * 4));
  for (auto& x : w.za) x = reinterpret_cast<__nv_bfloat16*>(take(rows_c * tc::kInvK * 2));
  w.yi = reinterpret_cast<float*>(take(rows_c * tc::kInvN * 4));
  w.part = reinterpret_cast<float*>(take(static_cast<size_t>(2 * num_sms) * tc::kBM * tc::kBN * 4));
  w.bytes = off;
  return w;
}

// D (m_pad x n) = A (m_pad x K, image planes) B^T on the tensor cores. When the grid of output
// tiles is small, K is split into groups whose folded partial sums a second kernel adds in
// group order.
cudaError_t launch_gemm(ar_ctx* ctx, __nv_bfloat16* const (&a)[3], size_t m_pad, int which, int terms, float* d,
                        float* part, cudaStream_t stream) {
  tc::GemmParams gp{};
  const int k = which == 0 ? tc::kFwdK : tc::kInvK;
  const int n = which == 0 ? tc::kFwdN : tc::kInvN;
  for (int pl = 0; pl < 3; ++pl) {
    gp.a[pl] = reinterpret_cast<const uint4*>(a[pl]);
    gp.b[pl] = ctx->tc_b[which][pl];
  }
  gp.err = ctx->d_err;
  gp.ldd = n;
  gp.chunks = k / tc::kBK;
  gp.terms = terms;
  int groups = 1;
  const int tiles128 = static_cast<int>(m_pad / tc::kBM) * (n / tc::kBN);
  while (groups * 2 <= gp.chunks && tiles128 * groups * 2 <= 2 * ctx->num_sms) groups *= 2;
  gp.chunks_per_group = gp.chunks / groups;
  // 256-wide tiles (half the MMA instructions and B-operand copies per flop) for the two-plane
  // split when every item is a single fold unit of at most four chunks and enough tiles remain
  const bool wide = terms == 3 && gp.chunks_per_group <= 4 && n % 256 == 0 &&
                    static_cast<long long>(m_pad / tc::kBM) * (n / 256) >= 2 * ctx->num_sms;
  const int bn = wide ? 256 : tc::kBN;
  const int tiles = static_cast<int>(m_pad / tc::kBM) * (n / bn);
  gp.d = groups > 1 ? part : d;
  gp.d_group = m_pad * static_cast<size_t>(n);
  gp.m_tiles = static_cast<int>(m_pad / tc::kBM);
  gp.n_tiles = n / bn;
  gp.groups = groups;
  // persistent: one CTA per SM (the kernel's shared memory allows one), items strided
  const int items = tiles * groups;
  if (wide)
    tc::split_gemm_kernel<256><<<std::min(items, ctx->num_sms), tc::kGemmThreads, tc::kGemmSmem, stream>>>(gp);
  else
    tc::split_gemm_kernel<128><<<std::min(items, ctx->num_sms), tc::kGemmThreads, tc::kGemmSmem, stream>>>(gp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || groups == 1) return e;
  const size_t n4 = gp.d_group / 4;
  tc::tc_reduce_kernel<<<2 * ctx->num_sms, 256, 0, stream>>>(reinterpret_cast<const float4*>(part),
                                                              reinterpret_cast<float4*>(d), n4, n4, groups);
  return cudaGetLastError();
}

template <int N_>
cudaError_t launch_tc(ar_ctx* ctx, const EventDesc& ev, int terms, size_t rows_f, long long chunk,
                      cudaStream_t stream) {
  constexpr int A = N_ / tc::kSub;
  const int S = ev.n_st, D = ev.n_dir;
  const long long pairs = static_cast<long long>(S) * D;
  const size_t rows_c = pad128(static_cast<size_t>(2 * A) * chunk);
  const TcWorkspace w = tc_layout(ctx->tc_ws, rows_f, rows_c, ctx->num_sms);
  const int planes = terms == 6 ? 3 : 2;
  const tc::SplitImage fimg{{w.fa[0], w.fa[1], w.fa[2]}, planes};
  const tc::SplitImage zimg{{w.za[0], w.za[1], w.za[2]}, planes};
  const bool prof = ctx->profiling;
  cudaError_t e;
  if (prof && (e = cudaEventRecord(ctx->ev[0], stream)) != cudaSuccess) return e;
  tc::tc_forward_pre_kernel<N_><<<2 * S, tc::kSub, 0, stream>>>(ev, fimg);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_gemm(ctx, w.fa, rows_f, 0, terms, w.xf, w.part, stream)) != cudaSuccess) return e;
  // per-bin inverses [2][N/4] float4, then the node scratch [n_f][8] float2
  const size_t solve_smem = 2 * sizeof(float4) * (N_ / 4) + sizeof(float2) * 8 * static_cast<size_t>(ev.n_f_layout);
  int solve_per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&solve_per_sm, tc::tc_solve_kernel<N_>, tc::kSolveThreads,
                                                         solve_smem)) != cudaSuccess)
    return e;
  const long long solve_slots = std::max(1, solve_per_sm) * static_cast<long long>(ctx->num_sms);
  for (long long p0 = 0; p0 < pairs; p0 += chunk) {
    const int np = static_cast<int>(std::min(chunk, pairs - p0));
    // several pairs per CTA share the per-bin inverse: just enough that the CTAs fit in one
    // wave of resident CTAs (a second, partial wave would double the time)
    const int ppc = static_cast<int>(
        std::max<long long>(1, std::min<long long>(tc::kSolvePairsMax, (np + solve_slots - 1) / solve_slots)));
    tc::tc_solve_kernel<N_><<<(np + ppc - 1) / ppc, tc::kSolveThreads, solve_smem, stream>>>(
        ev, reinterpret_cast<const float2*>(w.xf), zimg, p0, np, ppc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (prof && p0 == 0 && (e = cudaEventRecord(ctx->ev[1], stream)) != cudaSuccess) return e;
    if ((e = launch_gemm(ctx, w.za, pad128(static_cast<size_t>(2 * A) * np), 1, terms, w.yi, w.part, stream)) !=
        cudaSuccess)
      return e;
    if (prof && p0 == 0 && (e = cudaEventRecord(ctx->ev[2], stream)) != cudaSuccess) return e;
    tc::tc_inverse_post_kernel<N_><<<np, tc::kSub, 0, stream>>>(ev, reinterpret_cast<const float2*>(w.yi), p0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  tc::tc_residual_kernel<<<D, 128, 0, stream>>>(ev);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (prof && (e = cudaEventRecord(ctx->ev[3], stream)) != cudaSuccess) return e;
  return cudaSuccess;
}

}  // namespace

extern "C" {

ar_status ar_unfold_tc(ar_ctx* ctx, const ar_event* ev, const ar_outputs* out, int32_t split_terms, void* stream) {
  NvtxRange nvtx("ar_unfold_tc");
  if (!ctx) return AR_ERR_INVALID_ARG;
  if (split_terms != 3 && split_terms != 6)
    return fail(ctx, AR_ERR_INVALID_ARG, "split_terms=%d: 3 or 6", split_terms);
  ar_status st = check_event(ctx, ev, out);
  if (st != AR_OK) return st;
  const long long S = ev->n_stations, N = ev->n_samples;
  if (N == 1024 || N == 2048 || N == 4096) {
    if (S * N > kTcMaxStationSamples)
      return fail(ctx, AR_ERR_INVALID_ARG, "the tensor-core variant takes at most %lld station samples (S*N=%lld)",
                  kTcMaxStationSamples, S * N);
  }
  AR_CUDA(ctx, cudaSetDevice(ctx->device));
  Resolved rs;
  if ((st = resolve(ctx, ev->n_samples, ev->fs_hz, ev->pattern_id, ev->n_stations, &rs, layout_nf(ctx, ev))) !=
      AR_OK)
    return st;
  if ((st = resolve_dirs(ctx, ev->n_dirs)) != AR_OK) return st;
  {
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if ((st = build_tc_tables(ctx)) != AR_OK) return st;
  }
  const int A = ev->n_samples / tc::kSub;
  const long long pairs = S * ev->n_dirs;
  const long long chunk = std::min<long long>(pairs, std::max<long long>(1, kTcChunkSamples / N));
  const size_t rows_f = pad128(static_cast<size_t>(2 * A) * S);
  const size_t rows_c = pad128(static_cast<size_t>(2 * A) * chunk);
  const size_t need = tc_layout(nullptr, rows_f, rows_c, ctx->num_sms).bytes;
  if (need > ctx->tc_ws_bytes) {
    AR_CUDA(ctx, cudaDeviceSynchronize());
    cudaFree(ctx->tc_ws);
    ctx->tc_ws = nullptr;
    ctx->tc_ws_bytes = 0;
    AR_CUDA(ctx, cudaMalloc(&ctx->tc_ws, need));
    ctx->tc_ws_bytes = need;
  }
  const PatternDev& pat = ctx->patterns[ev->pattern_id];
  PathBuffers b{ctx->spec, ctx->dir_done, ctx->d_err, rs.lt->t1, rs.lt->wn, rs.binf};
  EventDesc desc = make_desc(b, pat.desc, pat.table, ev, out, rs.k_lo);
  if ((st = attach_patterns(ctx, ev, rs.k_lo, &desc)) != AR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int terms = split_terms;
  cudaError_t e = ev->n_samples == 1024   ? launch_tc<1024>(ctx, desc, terms, rows_f, chunk, s)
                  : ev->n_samples == 2048 ? launch_tc<2048>(ctx, desc, terms, rows_f, chunk, s)
                                          : launch_tc<4096>(ctx, desc, terms, rows_f, chunk, s);
  if (e != cudaSuccess) return fail(ctx, AR_ERR_CUDA, "tensor-core path launch failed: %s", cudaGetErrorString(e));
  if (ctx->profiling) {
    ctx->timed = true;
    ctx->timed_tc = true;
  }
  return AR_OK;
}

}  // extern "C"

// ---- batched launches over uneven events ---------------------------------------------------
//
// A plan groups the events of a launch by trace length. Per length class it holds a device
// copy of the events' descriptors (behind a BatchHeader), and one CUDA graph runs, per class,
// the copy of the descriptors from pinned host staging, the station kernel (grid-stride over
// all stations of the class) and the persistent unfold kernel (contiguous chunks of all pairs
// of the class, crossing event boundaries). Classes are chained with programmatic dependent
// launch, so the next class's kernels start on SMs as the previous class's CTAs retire. Two
// pinned staging buffers and two graph instances alternate, so the host can fill the next
// launch while the previous one runs.

namespace {

constexpr int kClasses = 3;
int class_of(int n) { return n == 1024 ? 0 : n == 2048 ? 1 : 2; }

constexpr int kTuneMax = 6;   // the batch autotuner tries 1..kTuneMax unfold CTAs per SM

}  // namespace

struct ar_batch {
  ar_ctx* ctx = nullptr;
  ar_batch_limits lim{};
  size_t desc_bytes = 0;                       // header + max_events descriptors
  unsigned char* d_desc[kClasses] = {};        // device descriptors per class
  unsigned char* h_stage[2][kClasses] = {};    // pinned staging, two sets
  float4* spec = nullptr;                      // station spectra of all events
  size_t spec_bytes = 0;
  unsigned* dir_done = nullptr;
  DirPre* dir_pre = nullptr;
  cudaGraphExec_t exec[2][2] = {};            // [staging set][with SNRs], built when first needed
  cudaEvent_t done[2] = {nullptr, nullptr};
  bool pending[2] = {false, false};
  int next = 0;
  int ctas_per_sm[kClasses] = {0, 0, 0};       // chosen unfold occupancy per class
  int max_ctas_per_sm[kClasses] = {0, 0, 0};
  int slab_direct[kClasses] = {0, 0, 0};       // corner slabs read from L2 where staging them costs occupancy
  int max_staged[kClasses] = {0, 0, 0};        // the most CTAs per SM with the slabs staged (0: they do not fit)
  int max_direct[kClasses] = {0, 0, 0};        // ... with the slabs read from L2
  bool tuned = false;
  float tune_ms[kTuneMax + 1] = {};            // graph time per candidate CTAs per SM (autotune, stage 1)
  float default_ms = 0.f, tuned_ms = 0.f;      // graph time of the untuned and of the chosen plan
  int candidates = 0;                          // plans the autotuner timed
};

namespace {

template <int N_>
PathParams batch_params(ar_batch* b, int c, int wait_prior) {
  PathParams pp{};
  pp.batch = reinterpret_cast<const BatchHeader*>(b->d_desc[c]);
  pp.err = b->ctx->d_err;
  pp.wait_prior = wait_prior;
  return pp;
}

// Each station kernel computes while the previous one runs but waits for it before writing
// its spectra, so the completion of the last one implies the completion of all of them.
template <int N_>
cudaError_t batch_station_launch(ar_batch* b, int c, cudaStream_t st) {
  using L = Layout<N_>;
  return launch_pdl(station_spectrum_kernel<N_>, std::min(b->lim.max_stations, 4 * b->ctx->num_sms),
                    SpectrumSmem<N_>::BLOCK,
                    SpectrumSmem<N_>::TOTAL, st, batch_params<N_>(b, c, 1));
}

// The first unfold kernel waits for the last station kernel (so for all of them); the later
// ones need not wait: the kernel before them launches its dependents only after its own wait.
template <int N_>
cudaError_t batch_unfold_launch(ar_batch* b, int c, int ctas_per_sm, int wait_prior, bool snr, cudaStream_t st) {
  using L = Layout<N_>;
  const int grid = ctas_per_sm * b->ctx->num_sms;
  const size_t smem = UnfoldSmem<N_>::total(b->lim.max_n_freq, b->slab_direct[c] != 0);
  return snr ? launch_pdl(unfold_kernel<N_, true>, grid, L::T, smem, st, batch_params<N_>(b, c, wait_prior))
             : launch_pdl(unfold_kernel<N_, false>, grid, L::T, smem, st, batch_params<N_>(b, c, wait_prior));
}

// capture the whole launch (descriptor copies, then per class the two kernels) into graph g;
// snr: with the unfold instantiation that computes pulse SNRs
ar_status batch_build_graph(ar_batch* b, int set, const int* ctas, bool snr, cudaGraphExec_t* out) {
  ar_ctx* ctx = b->ctx;
  cudaStream_t cs;
  AR_CUDA(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  for (int c = 0; c < kClasses && e == cudaSuccess; ++c)
    e = cudaMemcpyAsync(b->d_desc[c], b->h_stage[set][c], b->desc_bytes, cudaMemcpyHostToDevice, cs);
  // station kernels of every class, then the unfold kernels, longest traces first so that
  // the finest-grained work fills the last tail
  if (e == cudaSuccess) e = batch_station_launch<1024>(b, 0, cs);
  if (e == cudaSuccess) e = batch_station_launch<2048>(b, 1, cs);
  if (e == cudaSuccess) e = batch_station_launch<4096>(b, 2, cs);
  if (e == cudaSuccess) e = batch_unfold_launch<4096>(b, 2, ctas[2], 1, snr, cs);
  if (e == cudaSuccess) e = batch_unfold_launch<2048>(b, 1, ctas[1], 0, snr, cs);
  if (e == cudaSuccess) e = batch_unfold_launch<1024>(b, 0, ctas[0], 0, snr, cs);
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return fail(ctx, AR_ERR_CUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
  return AR_OK;
}

// fill staging set `set` with the descriptors of the events
ar_status batch_fill(ar_batch* b, int set, const ar_event* events, const ar_outputs* outs, int n) {
  ar_ctx* ctx = b->ctx;
  BatchHeader* hdr[kClasses];
  EventDesc* dsc[kClasses];
  for (int c = 0; c < kClasses; ++c) {
    hdr[c] = reinterpret_cast<BatchHeader*>(b->h_stage[set][c]);
    dsc[c] = const_cast<EventDesc*>(batch_events(hdr[c]));
    hdr[c]->n_events = 0;
    hdr[c]->total_stations = 0;
    hdr[c]->total_pairs = 0;
  }
  size_t spec_off = 0, dir_off = 0;
  long long stations = 0, dirs = 0;
  for (int i = 0; i < n; ++i) {
    const ar_event* ev = &events[i];
    ar_status st = check_event(ctx, ev, &outs[i]);
    if (st != AR_OK) return fail(ctx, st, "event %d: %s", i, ctx->last_error.c_str());
    Resolved rs;
    if ((st = validate_shape(ctx, ev->n_samples, ev->fs_hz, ev->pattern_id, &rs.k_lo)) != AR_OK)
      return fail(ctx, st, "event %d: %s", i, ctx->last_error.c_str());
    if (layout_nf(ctx, ev) > b->lim.max_n_freq)
      return fail(ctx, AR_ERR_INVALID_ARG, "event %d: its patterns have %d frequency nodes, plan allows %d", i,
                  layout_nf(ctx, ev), b->lim.max_n_freq);
    if ((st = get_len_tables(ctx, ev->n_samples, rs.k_lo, &rs.lt)) != AR_OK) return st;
    if ((st = get_bin_table(ctx, ev->n_samples, ev->fs_hz, ev->pattern_id, rs.k_lo, &rs.binf)) != AR_OK) return st;
    stations += ev->n_stations;
    dirs += ev->n_dirs;
    const size_t sb = spec_ws_bytes(ev->n_samples, ev->n_stations);
    if (stations > b->lim.max_stations || dirs > b->lim.max_dirs || spec_off + sb > b->spec_bytes)
      return fail(ctx, AR_ERR_BUDGET, "events exceed the plan (stations %lld/%d, directions %lld/%d)", stations,
                  b->lim.max_stations, dirs, b->lim.max_dirs);
    const int c = class_of(ev->n_samples);
    PathBuffers pb{reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(b->spec) + spec_off),
                   b->dir_done + dir_off, ctx->d_err, rs.lt->t1, rs.lt->wn, rs.binf, b->dir_pre + dir_off};
    const PatternDev& pat = ctx->patterns[ev->pattern_id];
    EventDesc d = make_desc(pb, pat.desc, pat.table, ev, &outs[i], rs.k_lo);
    if ((st = attach_patterns(ctx, ev, rs.k_lo, &d)) != AR_OK) return st;
    d.n_f_layout = b->lim.max_n_freq;   // the plan's shared-memory layout
    d.slab_direct = b->slab_direct[c];
    d.pair_begin = hdr[c]->total_pairs;
    d.station_begin = hdr[c]->total_stations;
    dsc[c][hdr[c]->n_events++] = d;
    hdr[c]->total_stations += ev->n_stations;
    hdr[c]->total_pairs += static_cast<long long>(ev->n_stations) * ev->n_dirs;
    spec_off += (sb + 255) / 256 * 256;
    dir_off += ev->n_dirs;
  }
  return AR_OK;
}

}  // namespace

extern "C" {

ar_status ar_batch_create(ar_ctx* ctx, const ar_batch_limits* lim, ar_batch** out) {
  if (!ctx) return AR_ERR_INVALID_ARG;
  if (!lim || !out) return fail(ctx, AR_ERR_INVALID_ARG, "limits and output must not be NULL");
  if (lim->max_events < 1 || lim->max_events > (1 << 16) || lim->max_stations < 1 || lim->max_dirs < 1 ||
      lim->max_n_freq < 2 || lim->max_n_freq > kMaxFreqNodes)
    return fail(ctx, AR_ERR_INVALID_ARG, "batch limits out of range");
  AR_CUDA(ctx, cudaSetDevice(ctx->device));
  ar_batch* b = new ar_batch;
  b->ctx = ctx;
  b->lim = *lim;
  b->desc_bytes = 16 + sizeof(EventDesc) * static_cast<size_t>(lim->max_events);
  b->spec_bytes = (sizeof(float4) * 1024 + sizeof(int2)) * static_cast<size_t>(lim->max_stations) +
                  512 * static_cast<size_t>(lim->max_events);
  auto cleanup = [&](ar_status st) {
    ar_batch_destroy(b);
    return st;
  };
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < kClasses && e == cudaSuccess; ++c) {
    e = cudaMalloc(&b->d_desc[c], b->desc_bytes);
    for (int set = 0; set < 2 && e == cudaSuccess; ++set) e = cudaMallocHost(&b->h_stage[set][c], b->desc_bytes);
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->spec, b->spec_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&b->dir_done, sizeof(unsigned) * lim->max_dirs);
  if (e == cudaSuccess) e = cudaMemset(b->dir_done, 0, sizeof(unsigned) * lim->max_dirs);
  if (e == cudaSuccess) e = cudaMalloc(&b->dir_pre, sizeof(DirPre) * lim->max_dirs);
  for (int set = 0; set < 2 && e == cudaSuccess; ++set) e = cudaEventCreateWithFlags(&b->done[set], cudaEventDisableTiming);
  if (e != cudaSuccess) return cleanup(fail(ctx, AR_ERR_OUT_OF_MEMORY, "batch allocation failed: %s", cudaGetErrorString(e)));
  for (int c = 0; c < kClasses; ++c) {
    for (int set = 0; set < 2; ++set) std::memset(b->h_stage[set][c], 0, b->desc_bytes);
    const void* fn = c == 0 ? reinterpret_cast<const void*>(unfold_kernel<1024, false>)
                     : c == 1 ? reinterpret_cast<const void*>(unfold_kernel<2048, false>)
                              : reinterpret_cast<const void*>(unfold_kernel<4096, false>);
    const int threads = c == 0 ? Layout<1024>::T : c == 1 ? Layout<2048>::T : Layout<4096>::T;
    const auto smem_of = [&](bool direct) {
      return c == 0 ? UnfoldSmem<1024>::total(lim->max_n_freq, direct)
             : c == 1 ? UnfoldSmem<2048>::total(lim->max_n_freq, direct)
                      : UnfoldSmem<4096>::total(lim->max_n_freq, direct);
    };
    const size_t sp_smem = c == 0 ? SpectrumSmem<1024>::TOTAL : c == 1 ? SpectrumSmem<2048>::TOTAL : SpectrumSmem<4096>::TOTAL;
    const void* sfn = c == 0 ? reinterpret_cast<const void*>(station_spectrum_kernel<1024>)
                      : c == 1 ? reinterpret_cast<const void*>(station_spectrum_kernel<2048>)
                               : reinterpret_cast<const void*>(station_spectrum_kernel<4096>);
    const size_t smem_max = c == 0 ? UnfoldSmem<1024>::total(kMaxFreqNodes)
                            : c == 1 ? UnfoldSmem<2048>::total(kMaxFreqNodes)
                                     : UnfoldSmem<4096>::total(kMaxFreqNodes);
    if ((e = c == 0   ? set_unfold_smem_limit<1024>(smem_max)
             : c == 1 ? set_unfold_smem_limit<2048>(smem_max)
                      : set_unfold_smem_limit<4096>(smem_max)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(sfn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sp_smem))) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->max_ctas_per_sm[c], fn, threads, smem_of(false))) !=
            cudaSuccess)
      return cleanup(fail(ctx, AR_ERR_CUDA, "kernel set-up failed: %s", cudaGetErrorString(e)));
    int per_sm_direct = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_direct, fn, threads, smem_of(true))) != cudaSuccess)
      return cleanup(fail(ctx, AR_ERR_CUDA, "kernel set-up failed: %s", cudaGetErrorString(e)));
    b->max_staged[c] = b->max_ctas_per_sm[c];
    b->max_direct[c] = per_sm_direct;
    if (per_sm_direct > b->max_ctas_per_sm[c]) {
      b->slab_direct[c] = 1;
      b->max_ctas_per_sm[c] = per_sm_direct;
    }
    if (b->max_ctas_per_sm[c] < 1) return cleanup(fail(ctx, AR_ERR_CUDA, "unfold kernel does not fit an SM"));
    b->ctas_per_sm[c] = b->max_ctas_per_sm[c];
  }
  for (int set = 0; set < 2; ++set) {
    ar_status st = batch_build_graph(b, set, b->ctas_per_sm, false, &b->exec[set][0]);
    if (st != AR_OK) return cleanup(st);
  }
  b->tuned = !ctx->cfg.autotune;
  *out = b;
  return AR_OK;
}

ar_status ar_batch_destroy(ar_batch* b) {
  if (!b) return AR_OK;
  cudaSetDevice(b->ctx->device);
  for (int set = 0; set < 2; ++set) {
    if (b->pending[set]) cudaEventSynchronize(b->done[set]);
    for (int v = 0; v < 2; ++v)
      if (b->exec[set][v]) cudaGraphExecDestroy(b->exec[set][v]);
    if (b->done[set]) cudaEventDestroy(b->done[set]);
  }
  for (int c = 0; c < kClasses; ++c) {
    cudaFree(b->d_desc[c]);
    for (int set = 0; set < 2; ++set) cudaFreeHost(b->h_stage[set][c]);
  }
  cudaFree(b->spec);
  cudaFree(b->dir_done);
  cudaFree(b->dir_pre);
  delete b;
  return AR_OK;
}

// Time the whole graph of staging set `set` with the given CTAs per SM per class (the classes'
// slab staging as b->slab_direct holds it): one untimed launch, then the mean of three.
static ar_status batch_time_plan(ar_batch* b, int set, const int* ctas, bool snr, cudaStream_t stream,
                                 cudaEvent_t t0, cudaEvent_t t1, float* ms_out) {
  ar_ctx* ctx = b->ctx;
  cudaGraphExec_t g = nullptr;
  ar_status st = batch_build_graph(b, set, ctas, snr, &g);
  if (st != AR_OK) return st;
  float ms_sum = 0.f;
  for (int rep = 0; rep < 4; ++rep) {
    AR_CUDA(ctx, cudaEventRecord(t0, stream));
    AR_CUDA(ctx, cudaGraphLaunch(g, stream));
    AR_CUDA(ctx, cudaEventRecord(t1, stream));
    AR_CUDA(ctx, cudaEventSynchronize(t1));
    float ms = 0.f;
    AR_CUDA(ctx, cudaEventElapsedTime(&ms, t0, t1));
    if (rep > 0) ms_sum += ms;
  }
  cudaGraphExecDestroy(g);
  ++b->candidates;
  *ms_out = ms_sum / 3.f;
  return AR_OK;
}

// Stage the corner slabs of class c in shared memory (direct = 0) or read them from L2 (1), in
// the plan and in the descriptors of staging set `set`.
static void batch_set_slabs(ar_batch* b, int set, int c, int direct) {
  b->slab_direct[c] = direct;
  BatchHeader* hdr = reinterpret_cast<BatchHeader*>(b->h_stage[set][c]);
  EventDesc* d = const_cast<EventDesc*>(batch_events(hdr));
  for (int i = 0; i < hdr->n_events; ++i) d[i].slab_direct = direct;
}

// Autotune, on the events of staging set `set` (their results are the same for every plan).
// Stage 1: every class at min(k, its most CTAs per SM) for k = 1..6, keep the fastest k.
// Stage 2: per class, longest traces first, the CTAs per SM (1..its most) and the corner-slab
// placement (staged in shared memory where it fits, or read from L2) with the other classes
// fixed at their current choice; keep what is fastest. Classes without events keep stage 1's.
// Then both graphs are rebuilt with the plan.
static ar_status batch_autotune(ar_batch* b, int set, bool snr, cudaStream_t stream) {
  ar_ctx* ctx = b->ctx;
  cudaEvent_t t0, t1;
  AR_CUDA(ctx, cudaEventCreate(&t0));
  AR_CUDA(ctx, cudaEventCreate(&t1));
  b->candidates = 0;
  ar_status st = batch_time_plan(b, set, b->ctas_per_sm, snr, stream, t0, t1, &b->default_ms);
  int best[kClasses];
  float best_ms = b->default_ms;
  for (int c = 0; c < kClasses; ++c) best[c] = b->ctas_per_sm[c];
  const int kmax = std::max(b->max_ctas_per_sm[0], std::max(b->max_ctas_per_sm[1], b->max_ctas_per_sm[2]));
  for (int k = 1; st == AR_OK && k <= kmax && k <= kTuneMax; ++k) {
    int ctas[kClasses];
    for (int c = 0; c < kClasses; ++c) ctas[c] = std::min(k, b->max_ctas_per_sm[c]);
    st = batch_time_plan(b, set, ctas, snr, stream, t0, t1, &b->tune_ms[k]);
    if (st == AR_OK && b->tune_ms[k] < best_ms) {
      best_ms = b->tune_ms[k];
      for (int c = 0; c < kClasses; ++c) best[c] = ctas[c];
    }
  }
  for (int c = 2; st == AR_OK && c >= 0; --c) {
    if (reinterpret_cast<const BatchHeader*>(b->h_stage[set][c])->total_pairs == 0) continue;
    const int direct0 = b->slab_direct[c];
    int best_direct = direct0;
    for (int direct = 0; st == AR_OK && direct <= 1; ++direct) {
      const int most = direct ? b->max_direct[c] : b->max_staged[c];
      if (most < 1) continue;
      batch_set_slabs(b, set, c, direct);
      for (int k = 1; st == AR_OK && k <= most && k <= kTuneMax; ++k) {
        if (k == best[c] && direct == direct0) continue;   // timed already
        int ctas[kClasses] = {best[0], best[1], best[2]};
        ctas[c] = k;
        float ms = 0.f;
        st = batch_time_plan(b, set, ctas, snr, stream, t0, t1, &ms);
        if (st == AR_OK && ms < best_ms) {
          best_ms = ms;
          best[c] = k;
          best_direct = direct;
        }
      }
    }
    batch_set_slabs(b, set, c, best_direct);
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (st != AR_OK) return st;
  b->tuned_ms = best_ms;
  for (int c = 0; c < kClasses; ++c) b->ctas_per_sm[c] = best[c];
  for (int s2 = 0; s2 < 2; ++s2) {
    if (b->pending[s2]) AR_CUDA(ctx, cudaEventSynchronize(b->done[s2]));
    b->pending[s2] = false;
    for (int v = 0; v < 2; ++v) {
      if (b->exec[s2][v]) cudaGraphExecDestroy(b->exec[s2][v]);
      b->exec[s2][v] = nullptr;
    }
    ar_status st2 = batch_build_graph(b, s2, b->ctas_per_sm, snr, &b->exec[s2][snr ? 1 : 0]);
    if (st2 != AR_OK) return st2;
  }
  b->tuned = true;
  return AR_OK;
}

ar_status ar_batch_run(ar_batch* b, const ar_event* events, const ar_outputs* outs, int32_t n_events,
                       void* stream) {
  NvtxRange nvtx("ar_batch_run");
  if (!b) return AR_ERR_INVALID_ARG;
  ar_ctx* ctx = b->ctx;
  if (!events || !outs || n_events < 1) return fail(ctx, AR_ERR_INVALID_ARG, "events and outputs must not be empty");
  if (n_events > b->lim.max_events)
    return fail(ctx, AR_ERR_BUDGET, "%d events exceed the plan's %d", n_events, b->lim.max_events);
  AR_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int set = b->next;
  if (b->pending[set]) AR_CUDA(ctx, cudaEventSynchronize(b->done[set]));   // its staging is free again
  b->pending[set] = false;
  ar_status st = batch_fill(b, set, events, outs, n_events);
  if (st != AR_OK) return st;
  bool snr = false;
  for (int i = 0; i < n_events; ++i) snr = snr || outs[i].snr != nullptr;
  if (!b->tuned) {
    if ((st = batch_autotune(b, set, snr, s)) != AR_OK) return st;
  }
  cudaGraphExec_t& g = b->exec[set][snr ? 1 : 0];
  if (!g && (st = batch_build_graph(b, set, b->ctas_per_sm, snr, &g)) != AR_OK) return st;
  AR_CUDA(ctx, cudaGraphLaunch(g, s));
  AR_CUDA(ctx, cudaEventRecord(b->done[set], s));
  b->pending[set] = true;
  b->next = set ^ 1;
  return AR_OK;
}

ar_status ar_batch_tuning(const ar_batch* b, int32_t* ctas_per_sm, float* candidate_ms) {
  if (!b || !ctas_per_sm) return AR_ERR_INVALID_ARG;
  for (int c = 0; c < kClasses; ++c) ctas_per_sm[c] = b->ctas_per_sm[c];
  if (candidate_ms)
    for (int k = 0; k < kTuneMax; ++k) candidate_ms[k] = b->tune_ms[k + 1];
  return AR_OK;
}

ar_status ar_batch_tuning_info(const ar_batch* b, ar_batch_plan_info* info) {
  if (!b || !info) return AR_ERR_INVALID_ARG;
  for (int c = 0; c < kClasses; ++c) {
    info->ctas_per_sm[c] = b->ctas_per_sm[c];
    info->slabs_staged[c] = b->slab_direct[c] ? 0 : 1;
    info->max_ctas_per_sm[c] = b->max_ctas_per_sm[c];
  }
  info->tuned = b->tuned && b->ctx->cfg.autotune ? 1 : 0;
  info->candidates = b->candidates;
  info->default_ms = b->default_ms;
  info->tuned_ms = b->tuned_ms;
  return AR_OK;
}

}  // extern "C"

// ---- serving: continuous batching of host-buffer requests -------------------------------
//
// ar_submit hands the server an event and its outputs in host memory. A server thread admits
// queued requests in arrival order while their device state (inputs, outputs) fits the state
// budget, copies their inputs to the device on one stream, runs them as one batch launch on a
// second stream and copies the outputs back on a third. With two launches in flight, requests
// that arrive while the GPU is busy are admitted into the next launch as memory frees up; its
// copies overlap the running launch. Each request's arithmetic does not depend on the batch it
// ran in, so its results are the same alone and in the mix, bit for bit.

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// first-fit allocator over one device buffer (256-byte granules), coalescing on free
struct Arena {
  unsigned char* base = nullptr;
  size_t size = 0;
  std::map<size_t, size_t> free_list;   // offset -> length
  size_t used = 0;
  void init(unsigned char* b, size_t n) {
    base = b;
    size = n;
    free_list.clear();
    free_list[0] = n;
    used = 0;
  }
  bool alloc(size_t n, size_t* off) {
    n = (n + 255) / 256 * 256;
    for (auto it = free_list.begin(); it != free_list.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n;
        const size_t at = it->first + n;
        free_list.erase(it);
        if (rest) free_list[at] = rest;
        used += n;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = (n + 255) / 256 * 256;
    used -= n;
    auto it = free_list.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_list.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_list.erase(nx);
    }
    if (it != free_list.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_list.erase(it);
      }
    }
  }
};

struct Request {
  uint64_t ticket = 0;
  ar_event ev{};        // host arrays
  ar_outputs out{};     // host arrays
  size_t state_bytes = 0;
  size_t off = 0;       // arena offset of its device state
  ar_event dev_ev{};
  ar_outputs dev_out{};
  int64_t t_submit = 0, t_done = 0;
  ar_status status = AR_ERR_NOT_READY;
};

struct Launch {
  std::vector<uint64_t> tickets;
  cudaEvent_t h2d = nullptr, comp = nullptr, d2h = nullptr;
  bool busy = false;
};

size_t req_state_bytes(const ar_event& ev, const ar_outputs& out) {
  const size_t S = ev.n_stations, D = ev.n_dirs, N = ev.n_samples;
  auto r = [](size_t x) { return (x + 255) / 256 * 256; };
  size_t b = r(S * 2 * N * 4) + r(S * 24) + r(S * 8) + r(D * 16);
  if (ev.station_pattern) b += r(S * 4);
  if (out.efield) b += r(D * S * 2 * N * 4);
  if (out.envelope) b += r(D * S * N * 4);
  b += r(D * S * 4) * 2 + r(D * S * 8) * 2 + r(D * 8) * 2 + r(D * S * 4);
  if (out.peak_time_fine_ns) b += r(D * S * 8);
  if (out.snr) b += r(D * S * 4);
  return b;
}

}  // namespace

struct ar_server {
  ar_ctx* ctx = nullptr;
  ar_server_config cfg{};
  ar_batch* plan = nullptr;
  unsigned char* dev_state = nullptr;
  Arena arena;
  cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
  std::vector<Launch> launches;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;                          // submitted, not admitted
  std::unordered_map<uint64_t, Request> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  std::string error;
};

namespace {

// device layout of one request's state inside the arena
void place_request(ar_server* sv, Request& r) {
  unsigned char* p = sv->arena.base + r.off;
  const size_t S = r.ev.n_stations, D = r.ev.n_dirs, N = r.ev.n_samples;
  auto take = [&](size_t n) {
    unsigned char* q = p;
    p += (n + 255) / 256 * 256;
    return q;
  };
  r.dev_ev = r.ev;
  r.dev_ev.traces = reinterpret_cast<const float*>(take(S * 2 * N * 4));
  r.dev_ev.pos_m = reinterpret_cast<const double*>(take(S * 24));
  r.dev_ev.t_start_ns = reinterpret_cast<const double*>(take(S * 8));
  r.dev_ev.dirs_rad = reinterpret_cast<const double*>(take(D * 16));
  if (r.ev.station_pattern) r.dev_ev.station_pattern = reinterpret_cast<const int32_t*>(take(S * 4));
  r.dev_out = ar_outputs{};
  if (r.out.efield) r.dev_out.efield = reinterpret_cast<float*>(take(D * S * 2 * N * 4));
  if (r.out.envelope) r.dev_out.envelope = reinterpret_cast<float*>(take(D * S * N * 4));
  r.dev_out.peak_idx = reinterpret_cast<int32_t*>(take(D * S * 4));
  r.dev_out.peak_amp = reinterpret_cast<float*>(take(D * S * 4));
  r.dev_out.peak_time_ns = reinterpret_cast<double*>(take(D * S * 8));
  r.dev_out.residual_ns = reinterpret_cast<double*>(take(D * S * 8));
  r.dev_out.t0_ns = reinterpret_cast<double*>(take(D * 8));
  r.dev_out.chi2 = reinterpret_cast<double*>(take(D * 8));
  r.dev_out.status = reinterpret_cast<uint32_t*>(take(D * S * 4));
  if (r.out.peak_time_fine_ns) r.dev_out.peak_time_fine_ns = reinterpret_cast<double*>(take(D * S * 8));
  if (r.out.snr) r.dev_out.snr = reinterpret_cast<float*>(take(D * S * 4));
}

cudaError_t copy_in(ar_server* sv, const Request& r) {
  const size_t S = r.ev.n_stations, D = r.ev.n_dirs, N = r.ev.n_samples;
  cudaError_t e = cudaMemcpyAsync(const_cast<float*>(r.dev_ev.traces), r.ev.traces, S * 2 * N * 4,
                                  cudaMemcpyHostToDevice, sv->s_h2d);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(const_cast<double*>(r.dev_ev.pos_m), r.ev.pos_m, S * 24, cudaMemcpyHostToDevice, sv->s_h2d);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(const_cast<double*>(r.dev_ev.t_start_ns), r.ev.t_start_ns, S * 8, cudaMemcpyHostToDevice,
                        sv->s_h2d);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(const_cast<double*>(r.dev_ev.dirs_rad), r.ev.dirs_rad, D * 16, cudaMemcpyHostToDevice,
                        sv->s_h2d);
  if (e == cudaSuccess && r.ev.station_pattern)
    e = cudaMemcpyAsync(const_cast<int32_t*>(r.dev_ev.station_pattern), r.ev.station_pattern, S * 4,
                        cudaMemcpyHostToDevice, sv->s_h2d);
  return e;
}

cudaError_t copy_out(ar_server* sv, const Request& r) {
  const size_t S = r.ev.n_stations, D = r.ev.n_dirs, N = r.ev.n_samples;
  struct Item { void* h; const void* d; size_t n; };
  const Item items[] = {{r.out.efield, r.dev_out.efield, D * S * 2 * N * 4},
                        {r.out.envelope, r.dev_out.envelope, D * S * N * 4},
                        {r.out.peak_idx, r.dev_out.peak_idx, D * S * 4},
                        {r.out.peak_amp, r.dev_out.peak_amp, D * S * 4},
                        {r.out.peak_time_ns, r.dev_out.peak_time_ns, D * S * 8},
                        {r.out.residual_ns, r.dev_out.residual_ns, D * S * 8},
                        {r.out.t0_ns, r.dev_out.t0_ns, D * 8},
                        {r.out.chi2, r.dev_out.chi2, D * 8},
                        {r.out.status, r.dev_out.status, D * S * 4},
                        {r.out.peak_time_fine_ns, r.dev_out.peak_time_fine_ns, D * S * 8},
                        {r.out.snr, r.dev_out.snr, D * S * 4}};
  for (const Item& it : items) {
    if (!it.h || !it.d) continue;
    cudaError_t e = cudaMemcpyAsync(it.h, it.d, it.n, cudaMemcpyDeviceToHost, sv->s_d2h);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// complete finished launches (lock held)
void harvest(ar_server* sv) {
  for (Launch& L : sv->launches) {
    if (!L.busy || cudaEventQuery(L.d2h) != cudaSuccess) continue;
    const int64_t t = now_ns();
    for (uint64_t tk : L.tickets) {
      Request& r = sv->reqs[tk];
      sv->arena.release(r.off, r.state_bytes);
      r.t_done = t;
      r.status = AR_OK;
    }
    L.tickets.clear();
    L.busy = false;
    sv->cv_done.notify_all();
  }
}

void fail_request(ar_server* sv, Request& r, ar_status st) {
  r.status = st;
  r.t_done = now_ns();
  sv->cv_done.notify_all();
}

void server_loop(ar_server* sv) {
  cudaSetDevice(sv->ctx->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    harvest(sv);
    Launch* slot = nullptr;
    for (Launch& L : sv->launches)
      if (!L.busy) { slot = &L; break; }
    std::vector<uint64_t> batch;
    if (slot) {
      NvtxRange nvtx("server admit");
      // admit in arrival order while the state fits the budget
      size_t stations = 0, dirs = 0;
      while (!sv->queue.empty() && static_cast<int>(batch.size()) < sv->cfg.max_batch_events) {
        Request& r = sv->reqs[sv->queue.front()];
        if (r.state_bytes > sv->arena.size) {   // can never fit: refuse
          sv->queue.pop_front();
          fail_request(sv, r, AR_ERR_BUDGET);
          continue;
        }
        if (stations + r.ev.n_stations > static_cast<size_t>(sv->cfg.max_batch_events) * sv->cfg.max_stations_per_event ||
            dirs + r.ev.n_dirs > static_cast<size_t>(sv->cfg.max_batch_events) * 256)
          break;
        size_t off = 0;
        if (!sv->arena.alloc(r.state_bytes, &off)) break;   // wait for memory
        r.off = off;
        place_request(sv, r);
        stations += r.ev.n_stations;
        dirs += r.ev.n_dirs;
        batch.push_back(r.ticket);
        sv->queue.pop_front();
      }
    }
    if (batch.empty()) {
      if (sv->stop && sv->queue.empty()) {
        bool idle = true;
        for (Launch& L : sv->launches) idle = idle && !L.busy;
        if (idle) break;
      }
      sv->cv_work.wait_for(lk, std::chrono::microseconds(50));
      continue;
    }
    // launch: inputs in, one batch run, outputs out
    NvtxRange nvtx("server launch (copies in, batch run, copies out)");
    std::vector<ar_event> evs;
    std::vector<ar_outputs> outs;
    cudaError_t e = cudaSuccess;
    for (uint64_t tk : batch) {
      const Request& r = sv->reqs[tk];
      if (e == cudaSuccess) e = copy_in(sv, r);
      evs.push_back(r.dev_ev);
      outs.push_back(r.dev_out);
    }
    ar_status st = AR_OK;
    if (e == cudaSuccess) e = cudaEventRecord(slot->h2d, sv->s_h2d);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sv->s_comp, slot->h2d, 0);
    if (e == cudaSuccess) st = ar_batch_run(sv->plan, evs.data(), outs.data(), static_cast<int32_t>(evs.size()), sv->s_comp);
    if (e == cudaSuccess && st == AR_OK) e = cudaEventRecord(slot->comp, sv->s_comp);
    if (e == cudaSuccess && st == AR_OK) e = cudaStreamWaitEvent(sv->s_d2h, slot->comp, 0);
    for (uint64_t tk : batch)
      if (e == cudaSuccess && st == AR_OK) e = copy_out(sv, sv->reqs[tk]);
    if (e == cudaSuccess && st == AR_OK) e = cudaEventRecord(slot->d2h, sv->s_d2h);
    if (e != cudaSuccess || st != AR_OK) {
      sv->error = e != cudaSuccess ? cudaGetErrorString(e) : sv->ctx->last_error;
      cudaStreamSynchronize(sv->s_h2d);
      cudaStreamSynchronize(sv->s_comp);
      cudaStreamSynchronize(sv->s_d2h);
      for (uint64_t tk : batch) {
        Request& r = sv->reqs[tk];
        sv->arena.release(r.off, r.state_bytes);
        fail_request(sv, r, e != cudaSuccess ? AR_ERR_CUDA : st);
      }
      continue;
    }
    slot->tickets = batch;
    slot->busy = true;
  }
}

}  // namespace

extern "C" {

ar_status ar_server_create(ar_ctx* ctx, const ar_server_config* cfg, ar_server** out) {
  if (!ctx) return AR_ERR_INVALID_ARG;
  if (!cfg || !out) return fail(ctx, AR_ERR_INVALID_ARG, "config and output must not be NULL");
  ar_server_config c = *cfg;
  if (c.state_budget_bytes == 0) c.state_budget_bytes = ctx->cfg.state_budget_bytes;
  if (c.max_batch_events < 1 || c.max_batch_events > 4096 || c.max_inflight < 1 || c.max_inflight > 2 ||
      c.max_stations_per_event < 1 || c.max_n_freq < 2 || c.max_n_freq > kMaxFreqNodes)
    return fail(ctx, AR_ERR_INVALID_ARG, "server config out of range");
  AR_CUDA(ctx, cudaSetDevice(ctx->device));
  ar_server* sv = new ar_server;
  sv->ctx = ctx;
  sv->cfg = c;
  auto cleanup = [&](ar_status st) {
    ar_server_destroy(sv);
    return st;
  };
  ar_batch_limits lim{c.max_batch_events, c.max_batch_events * c.max_stations_per_event, c.max_batch_events * 256,
                      c.max_n_freq};
  ar_status st = ar_batch_create(ctx, &lim, &sv->plan);
  if (st != AR_OK) return cleanup(st);
  cudaError_t e = cudaMalloc(&sv->dev_state, c.state_budget_bytes);
  if (e != cudaSuccess) return cleanup(fail(ctx, AR_ERR_OUT_OF_MEMORY, "state budget allocation failed: %s", cudaGetErrorString(e)));
  sv->arena.init(sv->dev_state, c.state_budget_bytes);
  if ((e = cudaStreamCreateWithFlags(&sv->s_h2d, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&sv->s_comp, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&sv->s_d2h, cudaStreamNonBlocking)) != cudaSuccess)
    return cleanup(fail(ctx, AR_ERR_CUDA, "stream creation failed: %s", cudaGetErrorString(e)));
  sv->launches.resize(c.max_inflight);
  for (Launch& L : sv->launches) {
    if ((e = cudaEventCreateWithFlags(&L.h2d, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&L.comp, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&L.d2h, cudaEventDisableTiming)) != cudaSuccess)
      return cleanup(fail(ctx, AR_ERR_CUDA, "event creation failed: %s", cudaGetErrorString(e)));
  }
  sv->worker = std::thread(server_loop, sv);
  *out = sv;
  return AR_OK;
}

ar_status ar_submit(ar_server* sv, const ar_event* ev, const ar_outputs* out, uint64_t* ticket) {
  if (!sv) return AR_ERR_INVALID_ARG;
  ar_ctx* ctx = sv->ctx;
  if (!ticket) return fail(ctx, AR_ERR_INVALID_ARG, "ticket must not be NULL");
  ar_status st = check_event(ctx, ev, out);
  if (st != AR_OK) return st;
  int k_lo = 0;
  if ((st = validate_shape(ctx, ev->n_samples, ev->fs_hz, ev->pattern_id, &k_lo)) != AR_OK) return st;
  if (layout_nf(ctx, ev) > sv->cfg.max_n_freq)
    return fail(ctx, AR_ERR_INVALID_ARG, "the event's patterns have %d frequency nodes, the server allows %d",
                layout_nf(ctx, ev), sv->cfg.max_n_freq);
  if (ev->n_stations > sv->cfg.max_stations_per_event || ev->n_dirs > 256)
    return fail(ctx, AR_ERR_BUDGET, "event larger than the server's per-event limits (%d stations, 256 directions)",
                sv->cfg.max_stations_per_event);
  Request r;
  r.ev = *ev;
  r.out = *out;
  r.state_bytes = req_state_bytes(*ev, *out);
  if (r.state_bytes > sv->arena.size)
    return fail(ctx, AR_ERR_BUDGET, "event state %zu B exceeds the state budget %zu B", r.state_bytes, sv->arena.size);
  r.t_submit = now_ns();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return fail(ctx, AR_ERR_INVALID_ARG, "server is shutting down");
    r.ticket = sv->next_ticket++;
    *ticket = r.ticket;
    sv->reqs.emplace(r.ticket, r);
    sv->queue.push_back(r.ticket);
  }
  sv->cv_work.notify_one();
  return AR_OK;
}

ar_status ar_poll(ar_server* sv, uint64_t ticket) {
  if (!sv) return AR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return fail(sv->ctx, AR_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
  return it->second.status;
}

ar_status ar_wait(ar_server* sv, uint64_t ticket, int32_t timeout_ms) {
  if (!sv) return AR_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return fail(sv->ctx, AR_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  while (it->second.status == AR_ERR_NOT_READY) {
    if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && it->second.status == AR_ERR_NOT_READY)
      return AR_ERR_TIMEOUT;
  }
  return it->second.status;
}

ar_status ar_ticket_times(ar_server* sv, uint64_t ticket, int64_t* submit_ns, int64_t* done_ns) {
  if (!sv || !submit_ns || !done_ns) return AR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return fail(sv->ctx, AR_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
  *submit_ns = it->second.t_submit;
  *done_ns = it->second.t_done;
  return it->second.status;
}

ar_status ar_ticket_release(ar_server* sv, uint64_t ticket) {
  if (!sv) return AR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return fail(sv->ctx, AR_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
  if (it->second.status == AR_ERR_NOT_READY) return fail(sv->ctx, AR_ERR_NOT_READY, "ticket still in flight");
  sv->reqs.erase(it);
  return AR_OK;
}

ar_status ar_server_destroy(ar_server* sv) {
  if (!sv) return AR_OK;
  if (sv->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->stop = true;
    }
    sv->cv_work.notify_all();
    sv->worker.join();
  }
  cudaSetDevice(sv->ctx->device);
  for (Launch& L : sv->launches) {
    if (L.h2d) cudaEventDestroy(L.h2d);
    if (L.comp) cudaEventDestroy(L.comp);
    if (L.d2h) cudaEventDestroy(L.d2h);
  }
  if (sv->s_h2d) cudaStreamDestroy(sv->s_h2d);
  if (sv->s_comp) cudaStreamDestroy(sv->s_comp);
  if (sv->s_d2h) cudaStreamDestroy(sv->s_d2h);
  ar_batch_destroy(sv->plan);
  cudaFree(sv->dev_state);
  delete sv;
  return AR_OK;
}

}  // extern "C"

// ---- allocation-free entry point ----------------------------------------------------------
//
// For callers that cannot allocate device memory at all: code that runs inside a host that
// forbids cudaMalloc after start-up (a real-time data-taking loop with a fixed memory map, a
// plug-in living in someone else's CUDA context and memory pool). ar_unfold_noalloc runs the
// same three kernels as ar_unfold, but every buffer the library needs beyond the caller's
// inputs and outputs -- the station spectra, the twiddle and frequency-cell tables, the error
// word -- lives in the file-scope array below. The array exists once per GPU that loads the
// library and stays allocated until the process exits.

namespace {

constexpr size_t kNoAllocScratchBytes = 4u << 20;          // 4 MiB per device
constexpr size_t kNoAllocTablesBytes = 112u << 10;         // err, counters, T1, WN, cells (with headroom)
constexpr long long kNoAllocMaxStationSamples = 983040;    // stations x samples per channel
constexpr int kNoAllocMaxDirs = 4096;                      // directions per event
constexpr int kNoAllocMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

struct NoAllocDevice {
  bool ready = false;
  unsigned char* scratch = nullptr;   // device address of g_noalloc_scratch on this device
  int num_sms = 0;
};
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

// failures are reported through the calling thread's message that ar_last_error(NULL) returns
ar_status noalloc_fail(ar_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_create_error = buf;
  return st;
}

#define AR_NA_CUDA(call)                                                                   \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return noalloc_fail(AR_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Twiddle and frequency-cell tables of one trace length, computed on the device in FP64
// (sincospi) and rounded once to float; the same definitions as the host tables of ar_unfold.
template <int N_>
__global__ void noalloc_tables_kernel(float2* t1, float2* wn, int2* binf, int k_lo, double fs, double f0, double df,
                                      int n_f) {
  using L = Layout<N_>;
  constexpr int N = L::N, M = L::M, Q = L::Q, P = L::P;
  constexpr int NT1 = 4 * Q * P + (L::SPLIT == 1 ? 8 * Q : 0);   // pass-1 twiddles, then pass 2's (c, u)
  const int total = NT1 + N + M;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    double s, c;
    if (i < NT1) {
      long t;
      if (i < 4 * Q * P) {
        const int r = i / (Q * P), mb = (i / P) % Q, ja = i % P;
        t = (static_cast<long>(k_lo + ja) * (r + 4 * mb)) % N;
      } else {
        const int w = (i - 4 * Q * P) % (4 * Q);
        t = i - 4 * Q * P < 4 * Q ? (static_cast<long>(k_lo / P) * P * w) % N : w;
      }
      sincospi(2.0 * static_cast<double>(t) / N, &s, &c);
      t1[i] = make_float2(static_cast<float>(c), static_cast<float>(s));
    } else if (i < NT1 + N) {
      const int t = i - NT1;
      sincospi(2.0 * static_cast<double>(t) / N, &s, &c);
      wn[t] = make_float2(static_cast<float>(c), static_cast<float>(-s));
    } else {
      const int j = i - NT1 - N, k = k_lo + j;
      const double f = __ddiv_rn(__dmul_rn(static_cast<double>(k), fs), static_cast<double>(N));
      if (!(f >= kBandLoHz && f <= kBandHiHz)) {
        binf[j] = make_int2(-1, 0);
        continue;
      }
      double u = __ddiv_rn(__dsub_rn(f, f0), df);
      if (u < 0.0) u = 0.0;
      if (u > static_cast<double>(n_f - 1)) u = static_cast<double>(n_f - 1);
      int cell = static_cast<int>(floor(u));
      if (cell > n_f - 2) cell = n_f - 2;
      binf[j] = make_int2(cell, __float_as_int(static_cast<float>(__dsub_rn(u, static_cast<double>(cell)))));
    }
  }
}

// once per device, with that device current: the device address of the scratch array
ar_status noalloc_setup(int dev, NoAllocDevice** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return noalloc_fail(AR_ERR_CUDA, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoAllocDevice& d = g_noalloc_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    AR_NA_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    AR_NA_CUDA(upload_pretwiddles());
    AR_NA_CUDA(cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t sp1 = SpectrumSmem<1024>::TOTAL;
    const size_t sp2 = SpectrumSmem<2048>::TOTAL;
    const size_t sp4 = SpectrumSmem<4096>::TOTAL;
    AR_NA_CUDA(cudaFuncSetAttribute(station_spectrum_kernel<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sp1)));
    AR_NA_CUDA(cudaFuncSetAttribute(station_spectrum_kernel<2048>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sp2)));
    AR_NA_CUDA(cudaFuncSetAttribute(station_spectrum_kernel<4096>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sp4)));
    AR_NA_CUDA(set_unfold_smem_limit<1024>(UnfoldSmem<1024>::total(kMaxFreqNodes)));
    AR_NA_CUDA(set_unfold_smem_limit<2048>(UnfoldSmem<2048>::total(kMaxFreqNodes)));
    AR_NA_CUDA(set_unfold_smem_limit<4096>(UnfoldSmem<4096>::total(kMaxFreqNodes)));
    d.scratch = static_cast<unsigned char*>(p);
    d.ready = true;
  }
  *out = &d;
  return AR_OK;
}

template <int N_>
ar_status noalloc_launch(NoAllocDevice& nd, const ar_pattern_desc* pd, const float* table, const ar_event* ev,
                         const ar_outputs* out, int k_lo, cudaStream_t stream) {
  using L = Layout<N_>;
  unsigned char* base = nd.scratch;
  PathBuffers b{};
  b.err = reinterpret_cast<unsigned*>(base);
  b.dir_done = reinterpret_cast<unsigned*>(base + 256);                       // 16 KiB
  float2* t1 = reinterpret_cast<float2*>(base + 256 + (16u << 10));           // 32 KiB
  static_assert(sizeof(float2) * (4 * L::Q * L::P + (L::SPLIT == 1 ? 8 * L::Q : 0)) <= (32u << 10), "T1 area");
  float2* wn = reinterpret_cast<float2*>(base + 256 + (48u << 10));           // 32 KiB
  int2* binf = reinterpret_cast<int2*>(base + 256 + (80u << 10));             // 8 KiB
  b.t1 = t1;
  b.wn = wn;
  b.binf = binf;
  b.spec = reinterpret_cast<float4*>(base + kNoAllocTablesBytes);
  // the error word must start at zero (the direction counters are zeroed by the first
  // kernel); the tables are rewritten by every call
  AR_NA_CUDA(cudaMemsetAsync(b.err, 0, sizeof(unsigned), stream));
  noalloc_tables_kernel<N_><<<40, 256, 0, stream>>>(t1, wn, binf, k_lo, ev->fs_hz, pd->f0_hz, pd->df_hz,
                                                     pd->n_freq);
  AR_NA_CUDA(cudaGetLastError());
  int per_sm = 0, per_sm_direct = 0;
  AR_NA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, unfold_kernel<N_, false>, L::T,
                                                           UnfoldSmem<N_>::total(pd->n_freq)));
  AR_NA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_direct, unfold_kernel<N_, false>, L::T,
                                                           UnfoldSmem<N_>::total(pd->n_freq, true)));
  EventDesc desc = make_desc(b, *pd, reinterpret_cast<const float2*>(table), ev, out, k_lo);
  if (per_sm_direct > per_sm) {   // corner slabs read from L2 where staging them costs occupancy
    desc.slab_direct = 1;
    per_sm = per_sm_direct;
  }
  if (per_sm < 1) return noalloc_fail(AR_ERR_CUDA, "unfold kernel N=%d does not fit an SM", N_);
  AR_NA_CUDA(launch_path<N_>(b.err, desc, per_sm * nd.num_sms, stream, nullptr));
  return AR_OK;
}

}  // namespace

extern "C" {

ar_status ar_unfold_noalloc(const ar_pattern_desc* pd, const float* table, const ar_event* ev,
                            const ar_outputs* out, void* stream) {
  NvtxRange nvtx("ar_unfold_noalloc");
  if (!pd || !table) return noalloc_fail(AR_ERR_INVALID_ARG, "pattern descriptor and table must not be NULL");
  if (reinterpret_cast<uintptr_t>(table) % 16 != 0)
    return noalloc_fail(AR_ERR_INVALID_ARG, "the VEL table must be 16-byte aligned");
  char why[256];
  if (pattern_desc_error(pd, why, sizeof why)) return noalloc_fail(AR_ERR_INVALID_ARG, "%s", why);
  // the checks ar_unfold makes, then the ones of the fixed scratch
  if (event_error(ev, out, why, sizeof why)) return noalloc_fail(AR_ERR_INVALID_ARG, "%s", why);
  if (ev->station_pattern)
    return noalloc_fail(AR_ERR_INVALID_ARG, "per-station patterns need a context (ar_unfold); station_pattern must be NULL");
  if (ev->n_stations < 1 || ev->n_dirs < 1 || ev->n_dirs > kNoAllocMaxDirs)
    return noalloc_fail(AR_ERR_INVALID_ARG, "n_stations must be >= 1 and n_dirs in [1, %d]", kNoAllocMaxDirs);
  if (ev->n_samples != 1024 && ev->n_samples != 2048 && ev->n_samples != 4096)
    return noalloc_fail(AR_ERR_UNSUPPORTED_N, "n_samples=%d: supported lengths are 1024, 2048, 4096",
                        ev->n_samples);
  if (static_cast<long long>(ev->n_stations) * ev->n_samples > kNoAllocMaxStationSamples)
    return noalloc_fail(AR_ERR_INVALID_ARG,
                        "n_stations x n_samples = %lld exceeds the fixed scratch of ar_unfold_noalloc "
                        "(at most %lld: 240 stations of 4096, 480 of 2048 or 960 of 1024 samples)",
                        static_cast<long long>(ev->n_stations) * ev->n_samples, kNoAllocMaxStationSamples);
  if (!(ev->fs_hz > 0.0) || !std::isfinite(ev->fs_hz)) return noalloc_fail(AR_ERR_INVALID_ARG, "fs_hz must be positive");
  int lo, cnt, hi;
  band_window(ev->n_samples, ev->fs_hz, &lo, &cnt, &hi);
  if (cnt < 1 || cnt > ev->n_samples / 4 || lo + ev->n_samples / 4 > ev->n_samples / 2 || 2 * hi >= ev->n_samples)
    return noalloc_fail(AR_ERR_INVALID_ARG, "fs=%g Hz: the 30-80 MHz band must fit N/4 bins below Nyquist",
                        ev->fs_hz);
  int dev = 0;
  AR_NA_CUDA(cudaGetDevice(&dev));
  NoAllocDevice* nd = nullptr;
  ar_status st = noalloc_setup(dev, &nd);
  if (st != AR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (ev->n_samples) {
    case 1024: return noalloc_launch<1024>(*nd, pd, table, ev, out, lo, s);
    case 2048: return noalloc_launch<2048>(*nd, pd, table, ev, out, lo, s);
    default: return noalloc_launch<4096>(*nd, pd, table, ev, out, lo, s);
  }
}

}  // extern "C"
