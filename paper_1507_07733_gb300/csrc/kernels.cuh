// kernels.cuh -- device side of the unfolding path (sm_103a).
//
//   station_spectrum_kernel  forward transform of each station's two channels, one complex
//                            N-point DFT of (v0 + i v1) per station, split into the two real
//                            channels' spectra; only the M = N/4 bins of the band window kept
//   unfold_kernel            per (station, direction) pair: 2x2 solve per bin, inverse transform
//                            of the one-sided (analytic) spectrum, E-field, envelope, peak; a
//                            persistent grid walks the pairs direction-major, and per (direction,
//                            pattern) key the VEL interpolation and the per-bin inverse are formed
//                            once in shared memory (corner slabs staged by TMA bulk copies or read
//                            from L2) and applied to each of the key's stations; the CTA that
//                            finishes a direction last computes that direction's FP64 plane-wave
//                            timing residual (per-direction completion counters)
//
// Transform layout. The band holds at most M = N/4 bins, k in [k_lo, k_lo + M). The inverse
// transform z[n] = sum_k Z[k] exp(2 pi i k n / N) is evaluated at n = 4m + r (r = 0..3) as
// four M-point transforms, each split as M = P * Q:
//   j = k - k_lo = ja + P jb,  m = mb + Q ma
//   z[4m + r] = sum_ja exp(2 pi i ((k_lo+ja) mod P) ma / P) *
//               [ T1[r][mb][ja] * sum_jb (Z[k_lo+ja+P jb] exp(2 pi i jb r / 4Q)) exp(2 pi i jb mb / Q) ]
//   T1[r][mb][ja] = exp(2 pi i (k_lo + ja)(r + 4 mb) / N)
// Pass 1 is a Q-point DFT per (polarisation, r, ja); pass 2 a P-point DFT per (r, mb). The
// output phase of the band offset is absorbed by rotating pass 2's input rows by k_lo mod P,
// so no per-sample phase is applied at the end, and thread t of pass 2 writes samples
// n = t + 4Q ma: every warp store is 128 contiguous bytes. At N = 2048, where one pass-2
// thread holds both polarisations, T1 is applied in pass 2 instead (see pass1_task).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "dft.cuh"

namespace aerafold {

constexpr unsigned kStSingular = 1u;
constexpr unsigned kStZenClamp = 2u;
constexpr unsigned kStBadDir = 4u;
constexpr unsigned kStBadPattern = 8u;

constexpr unsigned kErrTmaTimeout = 1u;     // a bounded mbarrier wait ran out
constexpr unsigned kErrBounds = 4u;         // (debug build) an index check failed; the access was skipped

// Index checks of the debug build (compiled with AR_DEBUG_BOUNDS): a failed check sets
// kErrBounds in the error word, which ar_sync reports as AR_ERR_DEVICE, and the caller skips
// the access instead of trapping. In the release build every check is the constant true.
#ifdef AR_DEBUG_BOUNDS
__device__ __forceinline__ bool in_bounds(bool ok, unsigned* err) {
  if (!ok && err) atomicOr(err, kErrBounds);
  return ok;
}
#else
__device__ __forceinline__ constexpr bool in_bounds(bool, unsigned*) { return true; }
#endif
constexpr unsigned long long kWaitLimitNs = 1000000000ull;   // 1 s
constexpr unsigned long long kTestWaitLimitNs = 1000000ull;   // 1 ms: the limit under PathParams::test_wait

// ---- shapes per trace length ------------------------------------------------------------

template <int N_>
struct Shape;
template <>
struct Shape<1024> { static constexpr int N = 1024, M = 256, Q = 16, P = 16; };
template <>
struct Shape<2048> { static constexpr int N = 2048, M = 512, Q = 32, P = 16; };
template <>
struct Shape<4096> { static constexpr int N = 4096, M = 1024, Q = 32, P = 32; };

template <int N_>
struct Layout : Shape<N_> {
  using S = Shape<N_>;
  static constexpr int T = 8 * S::P;                  // threads: one pass-1 task each
  static constexpr int SPLIT = T / (4 * S::Q);        // pass-2 threads per (r, mb): 1 or 2
  static constexpr int MIN_CTAS = S::N == 1024 ? 5 : 512 / T;   // resident CTAs per SM the registers must allow
  static constexpr int LDA = S::Q + 1;                // row stride of A (float2)
  static constexpr int PLN0 = S::P * LDA;
  static constexpr int PLN = PLN0 + ((4 - PLN0 % 16) + 16) % 16;   // plane stride, == 4 mod 16
  static constexpr int A_F2 = 8 * PLN;                // A: [pol][r][row][mb]; E aliases it
  static_assert(SPLIT == 1 || SPLIT == 2, "layout");
  static_assert(A_F2 >= 2 * S::M, "E must fit in A");
  // with SPLIT == 2, the |Y|^2 exchange between the two polarisations' threads, P x 4Q
  // floats, also reuses A once pass 2 has read it
  static_assert(2 * A_F2 >= S::P * 4 * S::Q, "the exchange must fit in A");
  // outputs staged behind E: 16M bytes of E (or the exchange), then 3N floats
  static_assert(sizeof(float2) * A_F2 >= 16 * S::M + 12 * S::N, "the output staging must fit in A");
  static_assert(T % 32 == 0 && S::M % T == 0, "layout");
};

// ---- PTX helpers: shared-memory addresses, mbarrier, bulk copy, timer -------------------

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the phase with the given parity to complete; false if it did not within limit_ns
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
  return true;
}
// 1-D bulk copy global -> shared completing on an mbarrier (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// hardware approximations (relative error of a few ulp): used where FP32 rounding of the
// result is far below the path's 1e-5 tolerance
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// 1-D bulk copy shared -> global (16-byte aligned, size % 16 == 0), tracked as a bulk group
__device__ __forceinline__ void tma_bulk_s2g(void* dst, const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until the committed bulk stores have finished reading shared memory
__device__ __forceinline__ void tma_bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// wait until the committed bulk stores are complete
__device__ __forceinline__ void tma_bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// programmatic dependent launch: let the next kernel in the stream start its prologue, and
// wait for the previous kernel's completion (both are no-ops without the launch attribute)
// atomic add with acquire-release semantics at GPU scope; returns the previous value
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait_prior() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---- events as the kernels see them ------------------------------------------------------

// One antenna pattern as the kernels see it: its table, its frequency cell per band bin at
// the event's (N, fs), and its axes.
struct PatternRef {
  const float2* table;     // [n_zen][n_az][n_f][4] VEL (c0p0, c0p1, c1p0, c1p1)
  const int2* binf;        // [M]: (.x = frequency cell or -1 outside the band, .y = bits of t_f)
  double zen0, dzen, az0, daz;
  int n_zen, n_az, n_f, pad;
};

struct DirPre;

// One event. A plain call passes it inline in the kernel parameters; a batch launch reads
// an array of them, behind a header, from device memory (so a captured graph can be
// replayed with new events after a copy into that memory).
struct EventDesc {
  const float* traces;     // [S][2][N]
  const double* pos;       // [S][3]
  const double* t_start;   // [S]
  const double* dirs;      // [D][2]
  float* efield;           // [D][S][2][N] or null
  float* envelope;         // [D][S][N] or null
  int* peak_idx;           // [D][S]
  float* peak_amp;         // [D][S]
  double* peak_time;       // [D][S]
  double* peak_fine;       // [D][S] sub-sample peak times, or null (then the residual uses peak_time)
  float* snr;              // [D][S] pulse SNR, or null; when given the residual weights stations by it
  unsigned* status;        // [D][S]
  double* residual;        // [D][S]
  double* t0;              // [D]
  double* chi2;            // [D]
  float4* spec;            // [S][M] station band spectra (library workspace)
  unsigned* dir_done;      // [D] pairs finished per direction (library workspace)
  DirPre* dir_pre;         // [D] per-direction cells and vectors (library workspace), or null
  const float2* table;     // [n_zen][n_az][n_f][4] VEL (c0p0, c0p1, c1p0, c1p1)
  const int2* binf;        // [M]: (.x = frequency cell or -1 outside the band, .y = bits of t_f)
  const float2* t1;        // [4][Q][P] pass-1 output twiddles; with SPLIT == 1 then [2][4Q] (c, u) of pass 2
  const float2* wn;        // [N] exp(-2 pi i t / N)
  const PatternRef* pats;  // with st_pat: the loaded patterns at this (N, fs), by pattern id
  const int* st_pat;       // [S] pattern id per station, or null: every station uses the fields here
  int2* st_walk;           // [S] with st_pat: (station, pattern index) in walk order, written by the station kernel
  double zen0, dzen, az0, daz, dt_ns, n_over_c;
  double inv_n_st;         // 1 / n_st (FP64, from the host): the fit's mean as a product
  long long pair_begin;    // first pair of the event in the launch's flattened pair space
  int station_begin;       // first station of the event in the launch's flattened station space
  int n_zen, n_az, n_f, n_st, n_dir, k_lo;
  int n_pats;
  int n_f_layout;          // frequency nodes the unfold kernel's shared memory is laid out for (>= any pattern's)
  int slab_direct;         // 1: the corner slabs are read from the table in L2, not staged by TMA
  int pad2;
};

struct BatchHeader {       // in device memory, followed by EventDesc[n_events] (16-byte aligned)
  int n_events;
  int total_stations;
  long long total_pairs;
};

__host__ __device__ inline const EventDesc* batch_events(const BatchHeader* h) {
  return reinterpret_cast<const EventDesc*>(reinterpret_cast<const unsigned char*>(h) + 16);
}

struct PathParams {
  const BatchHeader* batch;   // device batch, or null: the single event ev0
  unsigned* err;              // device error word
  const int* skip;            // if not null and *skip != 0 the kernel does nothing (a loop has converged)
  int wait_prior;             // wait for the previous kernel in the stream (its results are needed)
  // Test of the bounded-wait error path (ar_set_test_fault): nonzero makes every corner-slab
  // mbarrier expect 16 bytes more than its four bulk copies deliver, and its waits give up
  // after 1 ms, so the waits run out, the error word gets kErrTmaTimeout and the CTAs return.
  // The copies themselves are unchanged and in bounds. 0 in every other launch.
  int test_wait;
  EventDesc ev0;
};

// index of the event whose [begin, begin + count) range holds x (events sorted by begin)
template <typename F>
__device__ __forceinline__ int find_event(int n, long long x, F begin_of) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (begin_of(mid) <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Pattern of station s: an index into ev.pats, -1 for the event's own pattern (no per-station
// ids), or -2 for an id outside the loaded patterns (the pair's outputs are then zero).
__device__ __forceinline__ int station_pattern(const EventDesc& ev, int s) {
  if (!ev.st_pat) return -1;
  const int p = ev.st_pat[s];
  return (p >= 0 && p < ev.n_pats) ? p : -2;
}
// Station and pattern index at position k of an event's station walk. With per-station ids
// the stations are walked grouped by pattern (stable order, unknown ids last; the station
// kernel writes the order), so that a direction's stations of one antenna type are adjacent
// and share one per-bin inverse.
__device__ __forceinline__ int2 walk_station(const EventDesc& ev, int k) {
  if (ev.st_walk) return __ldcg(ev.st_walk + k);
  return make_int2(k, station_pattern(ev, k));
}
__device__ __forceinline__ PatternRef pattern_ref(const EventDesc& ev, int p) {
  if (p >= 0) return ev.pats[p];
  PatternRef r;
  r.table = ev.table;
  r.binf = ev.binf;
  r.zen0 = ev.zen0;
  r.dzen = ev.dzen;
  r.az0 = ev.az0;
  r.daz = ev.daz;
  r.n_zen = ev.n_zen;
  r.n_az = ev.n_az;
  r.n_f = ev.n_f;
  r.pad = 0;
  return r;
}

// copy an event descriptor word by word (whole CTA)
__device__ __forceinline__ void copy_event(EventDesc* dst, const EventDesc* src, int tid, int nthreads) {
  static_assert(sizeof(EventDesc) % 8 == 0, "descriptor size");
  const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(dst);
  for (int i = tid; i < static_cast<int>(sizeof(EventDesc) / 8); i += nthreads) d[i] = s[i];
}


// ---- K1: forward transform of the station voltages ---------------------------------------

// Radices of the M-point transforms (M = N/4) of the station kernel, in stage order.
template <int N_>
struct StationRadix;
template <>
struct StationRadix<1024> { static constexpr int R0 = 4, R1 = 8, R2 = 8; };
template <>
struct StationRadix<2048> { static constexpr int R0 = 8, R1 = 8, R2 = 8; };
template <>
struct StationRadix<4096> { static constexpr int R0 = 16, R1 = 8, R2 = 8; };

template <int N_>
struct SpectrumSmem {
  static constexpr int N = N_, M = N_ / 4;
  static constexpr int THREADS = 256;                              // the transform's threads
  static constexpr int BLOCK = THREADS + 32;                       // and one warp for the direction entries
  static constexpr size_t X0 = 0;                                  // [4][M] float2 (ping)
  static constexpr size_t X1 = X0 + sizeof(float2) * 4 * M;        // [4][M] float2 (pong)
  static constexpr size_t TW = X1 + sizeof(float2) * 4 * M;        // [M] exp(-2 pi i x / M)
  static constexpr size_t TOTAL = TW + sizeof(float2) * M;
};

// One Stockham stage of radix R over the four M-point transforms held in `in` ([4][M]):
// span Ns (product of the radices already done); output in natural order after the last.
template <int M, int R>
__device__ __forceinline__ void stockham_stage(const float2* __restrict__ in, float2* __restrict__ out,
                                               const float2* __restrict__ tw, int Ns, int tid, int nthreads) {
  constexpr int MR = M / R;
  for (int task = tid; task < 4 * MR; task += nthreads) {
    const int sub = task / MR, j = task % MR;
    const int k = j % Ns;
    const float2* src = in + sub * M + j;
    float2 v[R];
    static_for<0, R>([&](auto q) { v[q] = src[q * MR]; });
    if (Ns > 1) {
      const int step = k * (M / (Ns * R));                   // twiddle exp(-2 pi i q k / (Ns R))
      static_for<1, R>([&](auto q) { v[q] = cmul(v[q], tw[q * step]); });
    }
    dft<R, -1>(v);
    float2* dst = out + sub * M + (j / Ns) * Ns * R + k;
    static_for<0, R>([&](auto q) { dst[q * Ns] = v[q]; });
  }
}

// a part of direction d's per-direction entry (defined with the cells)
__device__ void precompute_direction(const EventDesc& ev, int d, int part, bool valid);

// One CTA per station of the launch. x[4m + r] (both channels packed as v0 + i v1) -> four
// M-point DFTs U_r by three Stockham stages, then Z[k] = sum_r W_N^{kr} U_r[k mod M] at the
// band bins and the split into the two channels' spectra.
template <int N_>
__global__ void __launch_bounds__(SpectrumSmem<N_>::BLOCK) station_spectrum_kernel(const __grid_constant__ PathParams prm) {
  using SM = SpectrumSmem<N_>;
  using RD = StationRadix<N_>;
  constexpr int N = N_, M = SM::M, T = SM::THREADS;
  static_assert(RD::R0 * RD::R1 * RD::R2 == M, "radices");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* x0 = reinterpret_cast<float2*>(smem_raw + SM::X0);   // x[4m + r] at [r][m]; later U_r
  float2* x1 = reinterpret_cast<float2*>(smem_raw + SM::X1);
  float2* tw = reinterpret_cast<float2*>(smem_raw + SM::TW);
  const int tid = threadIdx.x;
  pdl_launch_dependents();
  // threads [0, T) transform (their barriers are named barrier 1); the last warp forms the
  // per-direction entries meanwhile (directions s, s + S, ... of the event for station s)
  const auto sync = [] { asm volatile("bar.sync 1, %0;" ::"n"(SM::THREADS) : "memory"); };
  // a plain launch has one CTA per station; a batch launch walks the stations grid-stride
  const int total = prm.batch ? prm.batch->total_stations : prm.ev0.n_st;
  for (int gs = blockIdx.x; gs < total; gs += gridDim.x) {
  const EventDesc* ev = &prm.ev0;
  if (prm.batch) {
    const EventDesc* evs = batch_events(prm.batch);
    ev = evs + find_event(prm.batch->n_events, gs, [&](int e) { return static_cast<long long>(evs[e].station_begin); });
  }
  const int s = gs - ev->station_begin;
  if (!in_bounds(s >= 0 && s < ev->n_st, prm.err)) continue;   // (uniform over the CTA)
  if (tid >= T) {
    if (ev->dir_pre) {
      // the previous kernel in the stream may still read the entries: wait before writing.
      // Ten direction slots of three lanes (see precompute_direction); lanes 30, 31 idle.
      if (prm.wait_prior) pdl_wait_prior();
      const int lane = tid - T, slot = lane / 3, part = lane % 3;
      const int S = ev->n_st, D = ev->n_dir;
      for (int base = s; base < D; base += 10 * S) {   // warp-uniform trip count
        const int d = base + S * slot;
        precompute_direction(*ev, d, part, slot < 10 && d < D);
      }
    }
    continue;
  }

  const float4* v0 = reinterpret_cast<const float4*>(ev->traces + static_cast<size_t>(s) * 2 * N);
  const float4* v1 = v0 + N / 4;
  const float2* wn = ev->wn;
  for (int m = tid; m < M; m += T) {
    const float4 a = __ldg(v0 + m), b = __ldg(v1 + m);
    x0[0 * M + m] = make_float2(a.x, b.x);
    x0[1 * M + m] = make_float2(a.y, b.y);
    x0[2 * M + m] = make_float2(a.z, b.z);
    x0[3 * M + m] = make_float2(a.w, b.w);
    tw[m] = __ldg(wn + 4 * m);                               // exp(-2 pi i m / M)
  }
  sync();
  stockham_stage<M, RD::R0>(x0, x1, tw, 1, tid, T);
  sync();
  stockham_stage<M, RD::R1>(x1, x0, tw, RD::R0, tid, T);
  sync();
  stockham_stage<M, RD::R2>(x0, x1, tw, RD::R0 * RD::R1, tid, T);
  sync();
  const float2* U = x1;                                      // U_r[k'] at [r][k']
  // the previous kernel in the stream may still read these spectra: wait before writing them
  if (prm.wait_prior) pdl_wait_prior();
  if (s == 0)
    for (int d = tid; d < ev->n_dir; d += T) ev->dir_done[d] = 0u;
  if (ev->st_walk) {   // this station's position in the walk: stable by pattern, unknown ids last
    const int S = ev->n_st, np = ev->n_pats;
    const auto key = [&](int x) { const int p = station_pattern(*ev, x); return p < 0 ? np : p; };
    const int ks = key(s);
    int c = 0;
    for (int x = tid; x < S; x += T) {
      const int kx = key(x);
      c += (kx < ks || (kx == ks && x < s)) ? 1 : 0;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    int* part = reinterpret_cast<int*>(x0);   // free since the last Stockham stage
    if ((tid & 31) == 0) part[tid >> 5] = c;
    sync();
    if (tid == 0) {
      int rank = 0;
#pragma unroll
      for (int w = 0; w < T / 32; ++w) rank += part[w];
      if (in_bounds(rank >= 0 && rank < S, prm.err)) ev->st_walk[rank] = make_int2(s, ks == np ? -2 : ks);
    }
  }
  // combine the four decimated transforms at k and N - k, split the channels
  float4* out = ev->spec + static_cast<size_t>(s) * M;
  const int k_lo = ev->k_lo;
  for (int j = tid; j < M; j += T) {
    const int k = k_lo + j;
    const int kk = k % M, km = (M - kk) % M;
    const float2 w1 = __ldg(wn + k);                      // W_N^k; W_N^{2k}, W_N^{3k} by products
    const float2 w2 = cmul(w1, w1), w3 = cmul(w2, w1);
    float2 z = U[kk], zm = U[km];
    z = cadd(z, cmul(U[M + kk], w1));
    zm = cadd(zm, cmulc(U[M + km], w1));                 // W_N^{-kr} = conj
    z = cadd(z, cmul(U[2 * M + kk], w2));
    zm = cadd(zm, cmulc(U[2 * M + km], w2));
    z = cadd(z, cmul(U[3 * M + kk], w3));
    zm = cadd(zm, cmulc(U[3 * M + km], w3));
    const float2 sum = make_float2(z.x + zm.x, z.y - zm.y);   // Z[k] + conj Z[N-k]
    const float2 dif = make_float2(z.x - zm.x, z.y + zm.y);   // Z[k] - conj Z[N-k]
    out[j] = make_float4(0.5f * sum.x, 0.5f * sum.y, 0.5f * dif.y, -0.5f * dif.x);
  }
  sync();   // shared buffers free for the next station
  }
}

// ---- K3: fused per-pair unfold + per-direction residual ------------------------------------

struct DirInfo {
  int slab0, slab1, slab2, slab3;   // node offsets (units of n_f * 4 float2) of the 4 corners
  float w[4];                       // bilinear weights of the corners
  unsigned st;
  int pat;                          // the station pattern the cell belongs to (station_pattern)
};

// Per direction of a launch, formed once by the station kernel: the direction cell in the
// event's own pattern (events without station ids) and the unit vector toward the source.
struct DirPre {
  DirInfo cell;
  double n[3];
  double pad;
};

// Direction -> pattern cell (FP64, no fused multiply-adds) -> FP32 bilinear weights.
__device__ __forceinline__ DirInfo direction_cell(const PatternRef& p, double zen, double az) {
  DirInfo di;
  di.st = 0;
  di.pat = -1;
  // A direction has a cell when it is finite and its azimuth lies less than 2^52 azimuth
  // steps from az0 (beyond, one FP64 unit is a whole step). Below that bound the remainder
  // modulo n_az lands in [0, n_az]; the range test keeps every slab index in bounds.
  double ua = 0.0;
  bool has_cell = isfinite(zen) && isfinite(az);
  if (has_cell) {
    ua = __ddiv_rn(__dsub_rn(az, p.az0), p.daz);
    has_cell = fabs(ua) < 0x1p52;
  }
  if (has_cell) {
    ua = __dsub_rn(ua, __dmul_rn(double(p.n_az), floor(__ddiv_rn(ua, double(p.n_az)))));
    has_cell = ua >= 0.0 && ua <= double(p.n_az);
  }
  if (!has_cell) {   // every output of the direction's pairs is 0
    di.st = kStBadDir;
    di.slab0 = di.slab1 = di.slab2 = di.slab3 = 0;
    di.w[0] = di.w[1] = di.w[2] = di.w[3] = 0.f;
    return di;
  }
  double uz = __ddiv_rn(__dsub_rn(zen, p.zen0), p.dzen);
  if (uz < 0.0) { uz = 0.0; di.st |= kStZenClamp; }
  if (uz > double(p.n_zen - 1)) { uz = double(p.n_zen - 1); di.st |= kStZenClamp; }
  int iz = static_cast<int>(floor(uz));
  if (iz > p.n_zen - 2) iz = p.n_zen - 2;
  const double tz = __dsub_rn(uz, double(iz));
  int ia = static_cast<int>(floor(ua));
  const double ta = __dsub_rn(ua, double(ia));
  if (ia >= p.n_az) ia -= p.n_az;
  const int ia1 = ia + 1 == p.n_az ? 0 : ia + 1;
  di.slab0 = iz * p.n_az + ia;          // (iz,   ia)
  di.slab1 = (iz + 1) * p.n_az + ia;    // (iz+1, ia)
  di.slab2 = iz * p.n_az + ia1;         // (iz,   ia+1)
  di.slab3 = (iz + 1) * p.n_az + ia1;   // (iz+1, ia+1)
  const double uz0 = __dsub_rn(1.0, tz), ua0 = __dsub_rn(1.0, ta);
  di.w[0] = static_cast<float>(__dmul_rn(uz0, ua0));
  di.w[1] = static_cast<float>(__dmul_rn(tz, ua0));
  di.w[2] = static_cast<float>(__dmul_rn(uz0, ta));
  di.w[3] = static_cast<float>(__dmul_rn(tz, ta));
  return di;
}

// Pre-twiddles of pass 1 for the 1024- and 4096-sample layouts, exp(2 pi i jb r / 4Q) at
// [r][jb] (Q = 16 and 32), read with a warp-uniform r so that one copy of their pass-1 code
// serves all four r. Per-r copies made the 2048-sample scan 1 % faster alone, but a batch graph
// runs the three lengths' kernels side by side and larger code there cost more than it saved.
__constant__ float2 c_pre32[4][32];
__constant__ float2 c_pre16[4][16];

// Pass-1 loads of the 2048-sample layout with pre-twiddle, x[jb] = E_p[ja + P jb]
// exp(2 pi i jb R / 4Q) for one residue R as compile-time constants (R = 0 multiplies
// nothing), the caller branching on the warp-uniform r; the DFT after them stays one code path
// (four full copies of pass 1 made the kernel limited by instruction fetch). The output
// twiddle's band wrap is absorbed here: for sh = 1 the task's rows carry an extra factor
// exp(2 pi i (4 mb + r) / 4Q) = exp(2 pi i mb / Q) exp(2 pi i r / 4Q), a cyclic shift of the DFT
// input by one slot: slot jb reads E_p[ja + P (jb - 1)] with the slot's own pre-twiddle, and
// slot 0 reads E_p[ja + P (Q - 1)] turned by i^R.
template <int Q, int P, int R>
__device__ __forceinline__ void load_pre_twiddled_wrap(const float2* Ep, int ja, bool sh, float2 (&x)[Q]) {
  const int b = sh ? ja - P : ja;   // slot jb >= 1 reads b + P jb (always in [0, P Q))
  const float2 e0 = Ep[sh ? ja + P * (Q - 1) : ja];
  if constexpr (R == 0) {
    x[0] = e0;
  } else {
    const float2 t = twmul<R, 4, +1>(e0);
    x[0] = sh ? t : e0;
  }
  static_for<1, Q>([&](auto jb) {
    constexpr long JB = decltype(jb)::value;
    x[JB] = twmul<JB * R, 4 * Q, +1>(Ep[b + P * JB]);
  });
}

// Pass 1 for one (pol, r, ja): load E_p[ja + P jb], pre-twiddle, Q-point inverse DFT, output
// twiddle T1[r][mb][ja] = w0 v^mb with w0 = T1[r][0][ja], v = T1[0][1][ja] = exp(2 pi i (k_lo+ja) 4/N).
// The twiddles are formed in registers as w0 (v^4)^i v^j (mb = 4i + j): two table loads per
// task instead of Q, at most ten roundings deep (relative error ~1e-6, inside the path's 1e-5).
//
// With SPLIT == 1 each pass-2 thread holds both polarisations of one (r, mb), so the output
// twiddle moves there and is formed once for both: write k_lo + ja = P (f0 + sh) + i with
// i = (k_lo + ja) mod P the task's row and f0 = floor(k_lo / P). Then
//   T1[r][mb][ja] = exp(2 pi i (P f0 + i)(4 mb + r) / N) * [sh] exp(2 pi i (4 mb + r) / 4Q);
// the first factor depends on (r, mb, i) only and is applied in pass 2 (tau_i = c u^i with
// c = exp(2 pi i P f0 (4 mb + r) / N), u = exp(2 pi i (4 mb + r) / N)), the second is the
// one-slot input shift of load_pre_twiddled_wrap.
template <int N_>
__device__ __forceinline__ void pass1_task(const float2* Ep, int ja, int r, int k_lo, const float2* __restrict__ t1,
                                           float2 (&x)[Layout<N_>::Q]) {
  using L = Layout<N_>;
  constexpr int Q = L::Q, P = L::P;
  if constexpr (L::SPLIT == 1) {
    const bool sh = ja + k_lo % P >= P;
    switch (r) {   // warp-uniform
      case 0: load_pre_twiddled_wrap<Q, P, 0>(Ep, ja, sh, x); break;
      case 1: load_pre_twiddled_wrap<Q, P, 1>(Ep, ja, sh, x); break;
      case 2: load_pre_twiddled_wrap<Q, P, 2>(Ep, ja, sh, x); break;
      default: load_pre_twiddled_wrap<Q, P, 3>(Ep, ja, sh, x); break;
    }
    dft<Q, +1>(x);
    return;
  }
  static_assert(Q == 32 || Q == 16, "pre-twiddle tables exist for Q = 16 and 32");
  const float2 w0 = __ldg(t1 + (r * Q) * P + ja);   // issued early: used after the DFT
  const float2 v1 = __ldg(t1 + P + ja);
  static_for<0, Q>([&](auto jb) {
    constexpr int JB = decltype(jb)::value;
    const float2 e = Ep[ja + P * JB];
    if constexpr (JB == 0) {
      x[JB] = e;
    } else {
      x[JB] = cmul(e, Q == 32 ? c_pre32[r][JB] : c_pre16[r][JB]);
    }
  });
  dft<Q, +1>(x);
  const float2 v2 = cmul(v1, v1), v3 = cmul(v2, v1), v4 = cmul(v2, v2);
  float2 a = w0;
  static_for<0, Q / 4>([&](auto i) {
    constexpr int I = decltype(i)::value;
    x[4 * I] = cmul(x[4 * I], a);
    x[4 * I + 1] = cmul(x[4 * I + 1], cmul(a, v1));
    x[4 * I + 2] = cmul(x[4 * I + 2], cmul(a, v2));
    x[4 * I + 3] = cmul(x[4 * I + 3], cmul(a, v3));
    if constexpr (I + 1 < Q / 4) a = cmul(a, v4);
  });
}

// Frequency nodes a pattern may have (the per-node interpolation scratch lives in A).
constexpr int kMaxFreqNodes = 256;

template <int N_>
struct UnfoldSmem {
  using L = Layout<N_>;
  // byte offsets inside dynamic shared memory (all 16-byte aligned)
  static constexpr size_t A = 0;
  // per band bin the scaled inverse of the 2x2 VEL matrix of the current (direction,
  // pattern): [2][M] float4, (h00, h01) then (h10, h11)
  static constexpr size_t HINV = A + sizeof(float2) * L::A_F2;
  static constexpr size_t EV = HINV + 2 * sizeof(float4) * L::M;            // current EventDesc
  static constexpr size_t DIR = EV + ((sizeof(EventDesc) + 15) / 16) * 16;  // 1 DirInfo
  static constexpr size_t RED = DIR + ((sizeof(DirInfo) + 15) / 16) * 16;   // reductions
  static constexpr size_t BAR = RED + 20 * (L::T / 32) + 32;   // T/32 x (double, float, int, float) + flag
  static constexpr size_t SLAB = BAR + 16;   // 4 * n_f * 4 float2 (staged corner slabs)
  // the per-node values and slopes (8 float2 per node) are formed in A before the solve
  static_assert(sizeof(float2) * L::A_F2 >= sizeof(float2) * 8 * kMaxFreqNodes, "node scratch must fit in A");
  __host__ __device__ static size_t total(int n_f, bool direct = false) {
    return SLAB + (direct ? 0 : sizeof(float2) * 16 * n_f);
  }
};

// Sub-sample offset of the envelope maximum at sample k: the vertex of the parabola through
// (k-1, k, k+1), in FP64; 0 at the trace ends or without a strict maximum, clamped to +-1/2.
__device__ __forceinline__ double peak_offset(const float* env, int n, int k) {
  if (k <= 0 || k >= n - 1) return 0.0;
  const double a = env[k - 1], b = env[k], c = env[k + 1];
  const double second = __dadd_rn(__dsub_rn(a, __dmul_rn(2.0, b)), c);
  if (!(second < 0.0)) return 0.0;
  const double delta = __ddiv_rn(__dmul_rn(0.5, __dsub_rn(a, c)), second);
  return fmin(0.5, fmax(-0.5, delta));
}

// Pulse SNR of a pair (a variant; the paper defines no noise estimate): (peak / noise)^2 at
// the envelope maximum k, noise^2 the mean of env^2 over the samples more than n/16 from k;
// 0 when there are none or their mean is 0. Whole CTA over the envelope in shared memory:
// thread t sums samples t, t + T, ..., the warps combine in a fixed tree and thread 0 adds the
// warps in order; the result is thread 0's. red holds T/32 floats.
template <int T>
__device__ __forceinline__ float pair_snr(const float* env, int n, int k, float peak, float* red) {
  const int w = n / 16;
  float acc = 0.f;
  for (int i = threadIdx.x; i < n; i += T) {
    const int dd = i > k ? i - k : k - i;
    if (dd > w) acc = fmaf(env[i], env[i], acc);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  float snr = 0.f;
  if (threadIdx.x == 0) {
    float ss = red[0];
#pragma unroll
    for (int i = 1; i < T / 32; ++i) ss += red[i];
    const int count = n - (min(k + w, n - 1) - max(k - w, 0) + 1);
    if (count > 0 && ss > 0.f) snr = peak * peak / (ss / static_cast<float>(count));
  }
  return snr;
}

// Residual of direction d over all stations, by the whole CTA (FP64, deterministic order:
// station s is handled by thread s mod T, and partial sums are combined in a fixed tree).
template <int T>
__device__ __forceinline__ double block_sum_fixed(double v, double* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double t = red[0];
#pragma unroll
  for (int i = 1; i < T / 32; ++i) t += red[i];
  return t;
}

template <int T>
__device__ __forceinline__ void direction_residual(const EventDesc& p, int d, double* red) {
  static_assert(T / 32 >= 3, "red holds the direction vector");
  // the direction vector: precomputed by the station kernel, else by one thread here (FP64
  // is a small fraction of the FP32 rate) and shared through red (at least 4 doubles;
  // block_sum_fixed synchronises before reusing it)
  double nx, ny, nz;
  if (p.dir_pre) {
    nx = __ldcg(&p.dir_pre[d].n[0]);
    ny = __ldcg(&p.dir_pre[d].n[1]);
    nz = __ldcg(&p.dir_pre[d].n[2]);
  } else {
    if (threadIdx.x == 0) {
      const double zen = p.dirs[2 * d], az = p.dirs[2 * d + 1];
      double sz, cz, sa, ca;   // sincos: the same values as separate sin and cos, half the FP64 work
      sincos(zen, &sz, &cz);
      sincos(az, &sa, &ca);
      red[0] = __dmul_rn(sz, ca);
      red[1] = __dmul_rn(sz, sa);
      red[2] = cz;
    }
    __syncthreads();
    nx = red[0];
    ny = red[1];
    nz = red[2];
  }
  // The stations' peak times t_start + index * dt (FP64) are formed here, the direction's
  // stations in parallel, rather than by one thread per pair; with sub-sample times (formed
  // per pair) the fit uses those.
  const int* ip = p.peak_idx + static_cast<size_t>(d) * p.n_st;
  double* ptime = p.peak_time + static_cast<size_t>(d) * p.n_st;
  const double* fine = p.peak_fine ? p.peak_fine + static_cast<size_t>(d) * p.n_st : nullptr;
  const auto time_of = [&](int s) {
    return __dadd_rn(p.t_start[s], __dmul_rn(static_cast<double>(__ldcg(ip + s)), p.dt_ns));
  };
  // with SNRs the fit weights station s by w_s = snr (a variant; its timing variance taken
  // inversely proportional to the SNR): t0 = sum w d / sum w, chi2 = sum w r^2; unweighted
  // when there are none or they sum to 0
  const float* wp = p.snr ? p.snr + static_cast<size_t>(d) * p.n_st : nullptr;
  double acc = 0.0, accw = 0.0, accwd = 0.0;
  double ds0 = 0.0;   // t_s - tau_s of this thread's first station, kept for the second pass
  for (int s = threadIdx.x; s < p.n_st; s += T) {
    const double* x = p.pos + 3 * s;
    const double dot = __dadd_rn(__dadd_rn(__dmul_rn(nx, x[0]), __dmul_rn(ny, x[1])), __dmul_rn(nz, x[2]));
    const double ts = time_of(s);
    ptime[s] = ts;
    const double ds = __dadd_rn(fine ? __ldcg(fine + s) : ts, __dmul_rn(dot, p.n_over_c));   // t_s - tau_s
    if (s == threadIdx.x) ds0 = ds;
    acc = __dadd_rn(acc, ds);
    if (wp) {
      const double w = static_cast<double>(__ldcg(wp + s));
      accw = __dadd_rn(accw, w);
      accwd = __dadd_rn(accwd, __dmul_rn(w, ds));
    }
  }
  const double sum = block_sum_fixed<T>(acc, red);
  double sw = 0.0, swd = 0.0;
  if (wp) {
    sw = block_sum_fixed<T>(accw, red);
    swd = block_sum_fixed<T>(accwd, red);
  }
  const bool weighted = wp && sw > 0.0;
  const double mean = weighted ? __ddiv_rn(swd, sw) : __dmul_rn(sum, p.inv_n_st);
  double ss = 0.0;
  double* res = p.residual + static_cast<size_t>(d) * p.n_st;
  for (int s = threadIdx.x; s < p.n_st; s += T) {
    double ds = ds0;
    if (s != threadIdx.x) {
      const double* x = p.pos + 3 * s;
      const double dot = __dadd_rn(__dadd_rn(__dmul_rn(nx, x[0]), __dmul_rn(ny, x[1])), __dmul_rn(nz, x[2]));
      ds = __dadd_rn(fine ? __ldcg(fine + s) : time_of(s), __dmul_rn(dot, p.n_over_c));
    }
    const double r = __dsub_rn(ds, mean);
    res[s] = r;
    ss = weighted ? __fma_rn(__dmul_rn(static_cast<double>(__ldcg(wp + s)), r), r, ss) : __fma_rn(r, r, ss);
  }
  ss = block_sum_fixed<T>(ss, red);
  if (threadIdx.x == 0) {
    p.t0[d] = mean;
    p.chi2[d] = ss;
    p.dir_done[d] = 0u;   // ready for the next launch
  }
}

// Direction cell of pair (d, s) in the station's pattern (pattern index p from station_pattern).
__device__ __forceinline__ DirInfo pair_cell(const EventDesc& ev, int d, int p, PatternRef* pr_out) {
  const PatternRef pr = pattern_ref(ev, p);
  DirInfo di = direction_cell(pr, ev.dirs[2 * d], ev.dirs[2 * d + 1]);
  if (p == -2) {   // not a loaded pattern: no interpolation, every output of the pair is zero
    di.st = kStBadPattern;
    di.slab0 = di.slab1 = di.slab2 = di.slab3 = 0;
    di.w[0] = di.w[1] = di.w[2] = di.w[3] = 0.f;
  }
  di.pat = p;
  if (pr_out) *pr_out = pr;
  return di;
}

// Part `part` (0, 1, 2) of direction d's entry, by three lanes of one warp in parallel (each
// part is a chain of slow FP64 operations): 0 the cell, 1 and 2 the sine and cosine of the
// zenith and of the azimuth, combined into the source vector by lane part 1. valid: d is a
// direction of the event (all three lanes of a slot agree); the shuffles run regardless.
__device__ void precompute_direction(const EventDesc& ev, int d, int part, bool valid) {
  double sv = 0.0, cv = 0.0;
  if (valid && part == 0) {
    DirPre* dp = ev.dir_pre + d;
    dp->cell = ev.st_pat ? DirInfo{} : pair_cell(ev, d, -1, nullptr);
  } else if (valid) {
    sincos(ev.dirs[2 * d + (part - 1)], &sv, &cv);
  }
  // part 1 (zenith) takes the azimuth's sine and cosine from part 2, the next lane
  const double sa = __shfl_down_sync(0xffffffffu, sv, 1), ca = __shfl_down_sync(0xffffffffu, cv, 1);
  if (valid && part == 1) {
    DirPre* dp = ev.dir_pre + d;
    dp->n[0] = __dmul_rn(sv, ca);
    dp->n[1] = __dmul_rn(sv, sa);
    dp->n[2] = cv;
    dp->pad = 0.0;
  }
}

// The cell of direction d in the event's own pattern as the station kernel formed it (read
// through L2: it was written by the previous kernel).
__device__ __forceinline__ DirInfo load_cell(const DirPre* dp) {
  DirInfo c;
  c.slab0 = __ldcg(&dp->cell.slab0);
  c.slab1 = __ldcg(&dp->cell.slab1);
  c.slab2 = __ldcg(&dp->cell.slab2);
  c.slab3 = __ldcg(&dp->cell.slab3);
#pragma unroll
  for (int i = 0; i < 4; ++i) c.w[i] = __ldcg(&dp->cell.w[i]);
  c.st = __ldcg(&dp->cell.st);
  c.pat = __ldcg(&dp->cell.pat);
  return c;
}

// Whether a key's corner slabs are staged in shared memory by bulk copies (else read from
// the L2-resident table when the key's inverse is built).
__device__ __forceinline__ bool slab_staged(const EventDesc& ev, int p) { return p != -2 && !ev.slab_direct; }

// For a new (direction, pattern) key (thread 0 only): the key's direction cell into sdir and,
// when the slabs are staged, the bulk copies of the pattern's four corner slabs, completing
// the mbarrier's current phase.
// With pre (after the wait for the station kernel) the event's own pattern's cell is taken
// from the direction's precomputed entry instead of being formed here in FP64.
__device__ __forceinline__ void issue_key(const EventDesc& ev, int d, int p, DirInfo* sdir, float2* slab,
                                          uint64_t* bar, bool pre = false, unsigned* err = nullptr,
                                          unsigned extra_tx = 0) {
  const PatternRef pr = pattern_ref(ev, p);
  DirInfo di = (pre && p == -1 && ev.dir_pre) ? load_cell(ev.dir_pre + d) : pair_cell(ev, d, p, nullptr);
  const int cells = pr.n_zen * pr.n_az;
  if (!in_bounds(di.slab0 >= 0 && di.slab0 < cells && di.slab1 >= 0 && di.slab1 < cells && di.slab2 >= 0 &&
                     di.slab2 < cells && di.slab3 >= 0 && di.slab3 < cells,
                 err))
    di.st |= kStBadDir;   // (debug build) no corner is read; the key's outputs are zero
  *sdir = di;
  if (!slab_staged(ev, p)) return;
  const unsigned slab_bytes = static_cast<unsigned>(pr.n_f) * 4u * sizeof(float2);
  const size_t node = static_cast<size_t>(pr.n_f) * 4;
  mbar_arrive_expect_tx(bar, 4 * slab_bytes + extra_tx);
  tma_bulk_g2s(slab + 0 * node, pr.table + di.slab0 * node, slab_bytes, bar);
  tma_bulk_g2s(slab + 1 * node, pr.table + di.slab1 * node, slab_bytes, bar);
  tma_bulk_g2s(slab + 2 * node, pr.table + di.slab2 * node, slab_bytes, bar);
  tma_bulk_g2s(slab + 3 * node, pr.table + di.slab3 * node, slab_bytes, bar);
}

// Build the per-bin inverse of a key (whole CTA; A is free): the bilinear (zenith, azimuth)
// interpolation of the four corners per frequency node and its slope to the next node into A,
// then per band bin the linear interpolation in frequency, the 2x2 determinant test and the
// scaled inverse, H^-1 * 2/N (the 2/N of the one-sided inverse transform, Sec. 3), into hinv.
// Returns whether any bin of the band was singular. Bins outside the pattern's frequency
// range, singular bins and keys with a bad direction or pattern get a zero inverse.
// T: the CTA's threads; direct: the corners are read from the table (else from slab).
template <int N_, int T = Layout<N_>::T>
__device__ __forceinline__ bool build_inverse(const EventDesc& ev, int p, const DirInfo& di, const float2* slab,
                                              bool direct, float2* hn, float4* hinv, unsigned* err = nullptr) {
  using L = Layout<N_>;
  constexpr int M = L::M, NB = M / T;
  static_assert(M % T == 0, "bins per thread");
  constexpr float kScale = 2.0f / static_cast<float>(L::N);
  const int tid = threadIdx.x;
  const bool valid = (di.st & (kStBadDir | kStBadPattern)) == 0;
  const PatternRef pr = pattern_ref(ev, p);
  if (valid) {
    const int n_f = pr.n_f;
    const size_t node = static_cast<size_t>(n_f) * 4;
    const float2* c0 = pr.table + di.slab0 * node;
    const float2* c1 = pr.table + di.slab1 * node;
    const float2* c2 = pr.table + di.slab2 * node;
    const float2* c3 = pr.table + di.slab3 * node;
    const auto bilin = [&](int x) {
      float2 a, b, c, dd;
      if (direct) {
        a = __ldg(c0 + x);
        b = __ldg(c1 + x);
        c = __ldg(c2 + x);
        dd = __ldg(c3 + x);
      } else {
        a = slab[x];
        b = slab[node + x];
        c = slab[2 * node + x];
        dd = slab[3 * node + x];
      }
      float2 h;
      h.x = fmaf(di.w[3], dd.x, fmaf(di.w[2], c.x, fmaf(di.w[1], b.x, di.w[0] * a.x)));
      h.y = fmaf(di.w[3], dd.y, fmaf(di.w[2], c.y, fmaf(di.w[1], b.y, di.w[0] * a.y)));
      return h;
    };
    for (int x = tid; x < n_f * 4; x += T) {
      const int f = x >> 2, cp = x & 3;
      const float2 h = bilin(x);
      const float2 h1 = f + 1 < n_f ? bilin(x + 4) : h;
      hn[8 * f + cp] = h;
      hn[8 * f + 4 + cp] = csub(h1, h);
    }
  }
  __syncthreads();
  bool sing = false;
#pragma unroll 1
  for (int i = 0; i < NB; ++i) {
    const int j = tid + T * i;
    float4 h0 = make_float4(0.f, 0.f, 0.f, 0.f), h1 = h0;
    int2 bf = valid ? __ldg(pr.binf + j) : make_int2(-1, 0);
    if (!in_bounds(bf.x < pr.n_f - 1, err)) bf.x = -1;   // a cell past the last node pair
    if (bf.x >= 0) {
      const float tf = __int_as_float(bf.y);
      const float4* g = reinterpret_cast<const float4*>(hn + 8 * bf.x);
      const float4 h01 = g[0], h23 = g[1], g01 = g[2], g23 = g[3];   // value, slope
      float2 a = make_float2(fmaf(tf, g01.x, h01.x), fmaf(tf, g01.y, h01.y));    // H0t
      float2 b = make_float2(fmaf(tf, g01.z, h01.z), fmaf(tf, g01.w, h01.w));    // H0p
      float2 c = make_float2(fmaf(tf, g23.x, h23.x), fmaf(tf, g23.y, h23.y));    // H1t
      float2 dd = make_float2(fmaf(tf, g23.z, h23.z), fmaf(tf, g23.w, h23.w));   // H1p
      // Scale H by the power of two 2^(127 - e) that brings its largest component to [1, 2):
      // exact, so the test and the inverse below give the same bits as unscaled wherever the
      // unscaled forms neither overflow nor underflow, and they never do for |H| far from 1
      // (the test compares fourth powers of |H|). The inverse is scaled back at the end.
      const float hm = fmaxf(fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(b.x), fabsf(b.y))),
                             fmaxf(fmaxf(fabsf(c.x), fabsf(c.y)), fmaxf(fabsf(dd.x), fabsf(dd.y))));
      const int ex = min(max(static_cast<int>((__float_as_uint(hm) >> 23) & 0xffu), 1), 253);
      const float up = __uint_as_float(static_cast<unsigned>(254 - ex) << 23);    // 2^(127 - ex)
      a = make_float2(a.x * up, a.y * up);
      b = make_float2(b.x * up, b.y * up);
      c = make_float2(c.x * up, c.y * up);
      dd = make_float2(dd.x * up, dd.y * up);
      const float2 det = csub(cmul(a, dd), cmul(b, c));
      const float sc = sqrt_approx(cabs2(a) * cabs2(dd)) + sqrt_approx(cabs2(b) * cabs2(c));
      const float dd2 = cabs2(det);
      if (dd2 > 1e-12f * sc * sc) {
        // X / det = X conj(det) / |det|^2, times `up` for the scaling of H
        const float inv = kScale * rcp_approx(dd2) * up;
        const float2 x00 = cmulc(dd, det), x01 = cmulc(b, det), x10 = cmulc(c, det), x11 = cmulc(a, det);
        h0 = make_float4(x00.x * inv, x00.y * inv, -x01.x * inv, -x01.y * inv);
        h1 = make_float4(-x10.x * inv, -x10.y * inv, x11.x * inv, x11.y * inv);
      } else {
        sing = true;
      }
    }
    hinv[j] = h0;
    hinv[M + j] = h1;
  }
  return __syncthreads_or(sing);
}

// kSnr: the instantiation that can compute pulse SNRs (for events that request them); the
// other one carries none of that code, which costs the plain path time even when unused.
template <int N_, bool kSnr>
__global__ void __launch_bounds__(Layout<N_>::T, Layout<N_>::MIN_CTAS) unfold_kernel(const __grid_constant__ PathParams prm) {
  using L = Layout<N_>;
  using SM = UnfoldSmem<N_>;
  constexpr int N = L::N, M = L::M, Q = L::Q, P = L::P, T = L::T, LDA = L::LDA, PLN = L::PLN;
  constexpr int SPLIT = L::SPLIT;
  constexpr int NB = M / T;   // solve bins per thread
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* A = reinterpret_cast<float2*>(smem_raw + SM::A);
  float2* E = A;    // E[pol][j], consumed by pass 1 before A is written
  float2* hn = A;   // per-node VEL values and slopes while a key's inverse is built
  float4* hinv = reinterpret_cast<float4*>(smem_raw + SM::HINV);
  EventDesc* sev = reinterpret_cast<EventDesc*>(smem_raw + SM::EV);
  DirInfo* sdir = reinterpret_cast<DirInfo*>(smem_raw + SM::DIR);
  double* redd = reinterpret_cast<double*>(smem_raw + SM::RED);      // T/32 doubles
  float* redv = reinterpret_cast<float*>(redd + T / 32);             // T/32 floats
  int* redi = reinterpret_cast<int*>(redv + T / 32);                 // T/32 ints
  int* sflag = redi + T / 32;                                        // 1 int
  float* redw = reinterpret_cast<float*>(sflag + 1);                // T/32 floats (SNR noise sums)
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + SM::BAR);
  float2* slab = reinterpret_cast<float2*>(smem_raw + SM::SLAB);

  const int tid = threadIdx.x;

  // the launch's events and the contiguous chunk of its flattened pair space for this CTA
  const EventDesc* evs = prm.batch ? batch_events(prm.batch) : &prm.ev0;
  const int n_events = prm.batch ? prm.batch->n_events : 1;
  const long long total_pairs =
      prm.batch ? prm.batch->total_pairs : static_cast<long long>(prm.ev0.n_st) * prm.ev0.n_dir;
  const long long per = total_pairs / gridDim.x, rem = total_pairs % gridDim.x;
  const long long q0 = blockIdx.x * per + min(static_cast<long long>(blockIdx.x), rem);
  const long long q1 = q0 + per + (blockIdx.x < rem ? 1 : 0);
  if (q0 >= q1) {
    if (prm.wait_prior) pdl_wait_prior();
    pdl_launch_dependents();
    return;
  }
  const int e0 = find_event(n_events, q0, [&](int e) { return evs[e].pair_begin; });

  // walk state, identical in every thread: event e, direction d, position k of pair q in the
  // event's station walk, its station s and the station's pattern p (see walk_station)
  int e = e0, d, k;
  {
    const long long lq = q0 - evs[e0].pair_begin;
    d = static_cast<int>(lq / evs[e0].n_st);
    k = static_cast<int>(lq % evs[e0].n_st);
  }
  // The station spectra and the walk order come from an earlier kernel; the pattern,
  // directions and station ids do not, unless a skip flag (written by the previous kernel,
  // which may cancel the whole launch) marks a loop whose directions the previous kernel
  // computes. Without either, the first key's inverse is built before waiting for the
  // previous kernel. After the wait the next kernel in the stream may launch, so that a kernel
  // launched behind this one may rely on everything this one waited for.
  const bool early = prm.skip == nullptr && evs[e0].st_walk == nullptr;
  if (!early) {
    if (prm.wait_prior) pdl_wait_prior();
    pdl_launch_dependents();
    if (prm.skip && *prm.skip) return;
  }
  int s, p;
  {
    const int2 w = walk_station(evs[e0], k);
    s = w.x;
    p = w.y;
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    issue_key(evs[e0], d, p, sdir, slab, bar, false, prm.err, prm.test_wait ? 16u : 0u);
  }
  bool pending = slab_staged(evs[e0], p);   // slab copies to wait for before the next build
  __syncthreads();    // barrier initialised, first direction cell visible

  int cur_e = e0 - 1;        // event of the previous pair (none yet)
  int cur_d = -1;
  int cur_p = -3;
  int pairs_in_dir = 0;
  DirInfo di;
  bool key_sing = false;
  unsigned phase = 0;
  float4 vin[NB];            // the pair's station spectrum at this thread's bins (from L2)
  const auto load_spec = [&](const EventDesc& x, int st) {
    if (!in_bounds(st >= 0 && st < x.n_st, prm.err)) {
#pragma unroll
      for (int i = 0; i < NB; ++i) vin[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      return;
    }
    const float4* src = x.spec + static_cast<size_t>(st) * M + tid;
#pragma unroll
    for (int i = 0; i < NB; ++i) vin[i] = __ldcg(src + T * i);
  };
  for (long long q = q0; q < q1; ++q) {
    if (pending) {
      const unsigned long long limit = prm.test_wait ? kTestWaitLimitNs : kWaitLimitNs;
      const bool ok = mbar_wait_bounded(bar, phase, limit);
      if (__syncthreads_or(!ok)) {   // a bulk copy never completed: report, give it one more bounded wait, leave
        if (tid == 0) {
          atomicOr(prm.err, kErrTmaTimeout);
          mbar_wait_bounded(bar, phase, limit);
          tma_bulk_wait_all();
        }
        __syncthreads();
        return;
      }
      phase ^= 1u;
    }
    if (e != cur_e) {   // new event: its descriptor into shared memory
      copy_event(sev, evs + e, tid, T);
      __syncthreads();
    }
    const EventDesc& ev = *sev;
    const int S = ev.n_st;
    // the next pair of this CTA: next station, else next direction, else the next event
    const bool has_next = q + 1 < q1;
    int e_next = e, d_next = d, k_next = k + 1;
    if (k_next == S) {
      k_next = 0;
      if (++d_next == ev.n_dir) {
        d_next = 0;
        ++e_next;
      }
    }
    const bool dir_end = !has_next || e_next != e || d_next != d;
    const EventDesc& evn = e_next != e ? evs[e_next] : ev;
    // (the walk order may come from the previous kernel: not read before waiting for it)
    int2 w_next = make_int2(s, p);
    if (has_next && !(q == q0 && early)) w_next = walk_station(evn, k_next);
    if (e != cur_e || d != cur_d || p != cur_p) {
      // new direction or pattern: the inverse of every bin, shared by the key's stations. The
      // node scratch overlays A: the previous pair's staged outputs must have left it.
      di = *sdir;
      if (tid == 0) tma_bulk_wait_read();
      __syncthreads();
      key_sing = build_inverse<N_>(ev, p, di, slab, ev.slab_direct != 0, hn, hinv, prm.err);
      cur_e = e;
      cur_d = d;
      cur_p = p;
    }
    if (q == q0) {
      if (early) {
        if (prm.wait_prior) pdl_wait_prior();
        pdl_launch_dependents();
      }
      load_spec(ev, s);
      if (has_next && early) w_next = walk_station(evn, k_next);
    }
    const int s_next = w_next.x, p_next = w_next.y;

    // ---- 2x2 solve per bin: E = H^-1 V ----
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int j = tid + T * i;
      const float4 h0 = hinv[j], h1 = hinv[M + j];   // (h00, h01), (h10, h11)
      const float4 v = vin[i];                       // (V0, V1)
      float2 et, ep;
      et.x = fmaf(h0.z, v.z, fmaf(-h0.w, v.w, fmaf(h0.x, v.x, -h0.y * v.y)));
      et.y = fmaf(h0.z, v.w, fmaf(h0.w, v.z, fmaf(h0.x, v.y, h0.y * v.x)));
      ep.x = fmaf(h1.z, v.z, fmaf(-h1.w, v.w, fmaf(h1.x, v.x, -h1.y * v.y)));
      ep.y = fmaf(h1.z, v.w, fmaf(h1.w, v.z, fmaf(h1.x, v.y, h1.y * v.x)));
      E[j] = et;
      E[M + j] = ep;
    }
    __syncthreads();   // E complete; the slab buffer is free from here

    const bool next_key = has_next && (dir_end || p_next != p);
    if (tid == 0 && next_key) {   // the next key's direction cell and corner slabs
      fence_proxy_async_smem();
      issue_key(evn, d_next, p_next, sdir, slab, bar, true, prm.err, prm.test_wait ? 16u : 0u);
    }
    pending = next_key && slab_staged(evn, p_next);

    // ---- pass 1: Q-point DFTs per (pol, r, ja) ----
    {
      const int r = tid / (2 * P);          // warp-uniform
      const int pol = (tid / P) & 1;
      const int ja = tid % P;
      float2 x[Q];
      const float2* Ep = E + pol * M;
      pass1_task<N_>(Ep, ja, r, ev.k_lo, ev.t1, x);
      if (tid == 0) tma_bulk_wait_read();   // the previous pair's staged outputs have left A
      __syncthreads();   // every E read done: A may overwrite it
      const int row = (ev.k_lo + ja) % P;
      float2* dst = A + (pol * 4 + r) * PLN + row * LDA;
      static_for<0, Q>([&](auto mb) { dst[mb] = x[mb]; });
    }
    __syncthreads();

    // ---- pass 2: P-point DFTs, E-field, envelope, peak ----
    // Outputs are staged in shared memory behind E (bytes [16M, 64M) of A: e_theta, e_phi,
    // envelope, N floats each) and written by two bulk copies; with SPLIT == 2 the |Y|^2
    // exchange uses the first 16M bytes (where E was).
    const size_t pair = static_cast<size_t>(d) * S + s;
    // (debug build) the pair lies in the event's outputs; otherwise none of its outputs is written
    const bool pair_ok = in_bounds(e < n_events && d >= 0 && d < ev.n_dir && s >= 0 && s < S, prm.err);
    const bool traces = ev.efield != nullptr && pair_ok;
    const bool want_snr = kSnr && ev.snr != nullptr;
    const bool stage_env = traces || ev.peak_fine != nullptr || want_snr;   // read back by those
    float* stage = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(A) + 16 * M);
    float bv = -1.0f;
    int bi = 0;
    if constexpr (SPLIT == 1) {
      const int r = tid & 3, mb = tid >> 2;   // 4 mb + r == tid
      // the output twiddles of pass 1's rows, tau_i = c u^i (see pass1_task)
      const float2 c = __ldg(ev.t1 + 4 * Q * P + tid), u1 = __ldg(ev.t1 + 4 * Q * P + T + tid);
      float2 y0[P], y1[P];
      const float2* src0 = A + r * PLN + mb;
      const float2* src1 = A + (4 + r) * PLN + mb;
      static_for<0, P>([&](auto i) {
        y0[i] = src0[i * LDA];
        y1[i] = src1[i * LDA];
      });
      __syncthreads();   // every A read done: the staging area may overwrite it
      {
        const float2 u2 = cmul(u1, u1), u3 = cmul(u2, u1), u4 = cmul(u2, u2);
        float2 a = c;   // tau_{4I}
        static_for<0, P / 4>([&](auto ii) {
          constexpr int I = decltype(ii)::value;
          const float2 w1 = cmul(a, u1), w2 = cmul(a, u2), w3 = cmul(a, u3);
          y0[4 * I] = cmul(y0[4 * I], a);
          y1[4 * I] = cmul(y1[4 * I], a);
          y0[4 * I + 1] = cmul(y0[4 * I + 1], w1);
          y1[4 * I + 1] = cmul(y1[4 * I + 1], w1);
          y0[4 * I + 2] = cmul(y0[4 * I + 2], w2);
          y1[4 * I + 2] = cmul(y1[4 * I + 2], w2);
          y0[4 * I + 3] = cmul(y0[4 * I + 3], w3);
          y1[4 * I + 3] = cmul(y1[4 * I + 3], w3);
          if constexpr (I + 1 < P / 4) a = cmul(a, u4);
        });
      }
      dft<P, +1>(y0);
      dft<P, +1>(y1);
      static_for<0, P>([&](auto ma) {
        const int n = tid + T * ma;
        const float v = sqrt_approx(fmaf(y0[ma].x, y0[ma].x, y0[ma].y * y0[ma].y) + cabs2(y1[ma]));
        if (traces) {
          stage[n] = y0[ma].x;
          stage[N + n] = y1[ma].x;
        }
        if (stage_env) stage[2 * N + n] = v;
        if (v > bv) { bv = v; bi = n; }
      });
    } else {
      constexpr int TQ = 4 * Q;
      const int pol = tid / TQ;             // warp-uniform
      const int tq = tid % TQ;
      const int r = tq & 3, mb = tq >> 2;
      float2 y[P];
      const float2* src = A + (pol * 4 + r) * PLN + mb;
      static_for<0, P>([&](auto i) { y[i] = src[i * LDA]; });
      __syncthreads();   // every A read done: the exchange and the staging area may overwrite it
      dft<P, +1>(y);
      float pw[P];
      static_for<0, P>([&](auto ma) {
        pw[ma] = cabs2(y[ma]);
        if (traces) stage[pol * N + tq + TQ * ma] = y[ma].x;
      });
      // the theta threads publish the powers of samples ma in [P/2, P), the phi threads those
      // of [0, P/2); each side then forms the envelope of the half it keeps ([P][TQ] floats)
      float* xch = reinterpret_cast<float*>(A);
      if (pol == 0) {
        static_for<P / 2, P>([&](auto ma) { xch[ma * TQ + tq] = pw[ma]; });
      } else {
        static_for<0, P / 2>([&](auto ma) { xch[ma * TQ + tq] = pw[ma]; });
      }
      __syncthreads();
      if (pol == 0) {
        static_for<0, P / 2>([&](auto ma) {
          const float v = sqrt_approx(pw[ma] + xch[ma * TQ + tq]);
          if (stage_env) stage[2 * N + tq + TQ * ma] = v;
          if (v > bv) { bv = v; bi = tq + TQ * ma; }
        });
      } else {
        static_for<P / 2, P>([&](auto ma) {
          const float v = sqrt_approx(pw[ma] + xch[ma * TQ + tq]);
          if (stage_env) stage[2 * N + tq + TQ * ma] = v;
          if (v > bv) { bv = v; bi = tq + TQ * ma; }
        });
      }
    }
    if (has_next) load_spec(evn, s_next);   // in flight through the pair's end
    // peak: max value, lowest index on ties
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if ((tid & 31) == 0) { redv[tid >> 5] = bv; redi[tid >> 5] = bi; }
    if (traces) fence_proxy_async_smem();   // each thread's staged writes, visible to the bulk copy
    __syncthreads();
    ++pairs_in_dir;
    if (tid == 0 && traces) {   // the staged E-field (both components) and envelope to global memory
      tma_bulk_s2g(ev.efield + pair * 2 * N, stage, 2 * N * sizeof(float));
      if (ev.envelope) tma_bulk_s2g(ev.envelope + pair * N, stage + 2 * N, N * sizeof(float));
      tma_bulk_commit();
    }
    float snr = 0.f;
    if (want_snr) {   // every thread takes the pair's peak from the per-warp maxima (as thread 0 does below)
      float pv = redv[0];
      int pk = redi[0];
#pragma unroll
      for (int w = 1; w < T / 32; ++w) {
        if (redv[w] > pv || (redv[w] == pv && redi[w] < pk)) { pv = redv[w]; pk = redi[w]; }
      }
      if (pv < 0.f) { pv = 0.f; pk = 0; }
      snr = pair_snr<T>(stage + 2 * N, N, pk, pv, redw);
    }
    if (tid == 0 && pair_ok) {
#pragma unroll
      for (int w = 1; w < T / 32; ++w) {
        if (redv[w] > bv || (redv[w] == bv && redi[w] < bi)) { bv = redv[w]; bi = redi[w]; }
      }
      if (bv < 0.f) { bv = 0.f; bi = 0; }
      ev.peak_idx[pair] = bi;
      ev.peak_amp[pair] = bv;   // the peak time is formed with the direction's residual
      if (ev.peak_fine)
        ev.peak_fine[pair] =
            __dadd_rn(ev.t_start[s], __dmul_rn(__dadd_rn(static_cast<double>(bi), peak_offset(stage + 2 * N, N, bi)),
                                               ev.dt_ns));
      ev.status[pair] = di.st | (key_sing ? kStSingular : 0u);
      if (want_snr) ev.snr[pair] = snr;
    }
    if (tid == 0 && dir_end) {   // publish this CTA's pairs of direction d; the last CTA does the residual
      // one acquire-release add: it releases this thread's outputs of the direction (the
      // only ones the residual reads) and acquires every other CTA's; the barrier below
      // passes them on to the CTA's other threads
      *sflag = 0;
      if (pair_ok) {
        const unsigned before = atom_add_acq_rel(ev.dir_done + d, static_cast<unsigned>(pairs_in_dir));
        *sflag = (before + pairs_in_dir == static_cast<unsigned>(S)) ? 1 : 0;
      }
    }
    if (dir_end) {
      pairs_in_dir = 0;
      __syncthreads();
      if (*sflag) direction_residual<T>(ev, d, redd);
    }
    __syncthreads();   // A, reductions and the event copy free for the next pair
    e = e_next;
    d = d_next;
    k = k_next;
    s = s_next;
    p = p_next;
  }
  if (tid == 0) tma_bulk_wait_all();
}

// ---- iterative reconstruction (Sec. 2): voltage-maximum timing, plane-wave fit -------------

struct ReconState {        // device memory, one per ar_reconstruct call
  double dir[2];           // direction the next unfold uses (zenith, azimuth)
  double t0;
  double chi2;
  int converged;           // set when the direction stops changing (or the fit fails)
  int iterations;          // unfold iterations whose results were fitted
  int failed;              // the first fit found no direction
  int pad;
};

struct FitParams {
  const double* pos;       // [S][3]
  const double* times;     // [S] station times to fit (voltage maxima, or the unfold's peak times)
  const int* idx;          // [S] the sample indices behind those times
  int* prev_idx;           // [S] the indices of the previous fit (updated here)
  ReconState* st;
  double* history;         // [(max_iter + 1)][2] or null
  double n_over_c, tol_rad;
  int n_st, iteration;     // iteration 0 fits the voltage maxima
};

// argmax_n v0[n]^2 + v1[n]^2 per station (FP64 squares, lowest index on ties); one CTA per station
__global__ void __launch_bounds__(256) voltage_peak_kernel(const float* traces, const double* t_start, int n,
                                                           double dt_ns, int* idx, double* t_ns) {
  const int s = blockIdx.x, tid = threadIdx.x;
  const float* v0 = traces + static_cast<size_t>(s) * 2 * n;
  const float* v1 = v0 + n;
  double bv = -1.0;
  int bi = 0;
  for (int j = tid; j < n; j += 256) {
    const double a = v0[j], b = v1[j];
    const double pw = __dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b));
    if (pw > bv) { bv = pw; bi = j; }
  }
  __shared__ double rv[8];
  __shared__ int ri[8];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, bv, off);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
  }
  if ((tid & 31) == 0) { rv[tid >> 5] = bv; ri[tid >> 5] = bi; }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < 8; ++w)
      if (rv[w] > bv || (rv[w] == bv && ri[w] < bi)) { bv = rv[w]; bi = ri[w]; }
    idx[s] = bi;
    t_ns[s] = __dadd_rn(t_start[s], __dmul_rn(static_cast<double>(bi), dt_ns));
  }
}

__device__ __forceinline__ double det3(const double (&a)[3][3]) {
  return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
         a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
}

// Least-squares plane wave t_s = t0 - n.x_s n_refr / c: linear in (t0, nx, ny) for a fixed nz,
// repeated four times with nz from the previous solution (nz = 1 first). One CTA of 128
// threads, FP64, sums in a fixed order. Also decides convergence and the residual chi2.
__global__ void __launch_bounds__(128) plane_fit_kernel(FitParams p) {
  ReconState* st = p.st;
  if (st->converged) return;
  const int tid = threadIdx.x;
  __shared__ double red[4][10];
  __shared__ double sol[4];
  __shared__ int same_s;
  // do the station indices repeat those of the previous fit?
  int diff = 0;
  if (p.iteration > 0)
    for (int s = tid; s < p.n_st; s += 128) diff |= p.idx[s] != p.prev_idx[s];
  const int any_diff = __syncthreads_or(diff);
  for (int s = tid; s < p.n_st; s += 128) p.prev_idx[s] = p.idx[s];
  if (tid == 0) same_s = p.iteration > 0 && !any_diff;
  const double k = p.n_over_c;
  double nz = 1.0;
  bool ok = true;
  for (int pass = 0; pass < 4 && ok; ++pass) {
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // n, Sx, Sy, Sxx, Sxy, Syy, Sy_t, Sx_t, Sy_t(y)
    for (int s = tid; s < p.n_st; s += 128) {
      const double x = p.pos[3 * s], y = p.pos[3 * s + 1], z = p.pos[3 * s + 2];
      const double yt = __dadd_rn(p.times[s], __dmul_rn(__dmul_rn(k, nz), z));
      v[0] += 1.0; v[1] += x; v[2] += y; v[3] += x * x; v[4] += x * y; v[5] += y * y;
      v[6] += yt; v[7] += x * yt; v[8] += y * yt;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      double t = v[i];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
      if ((tid & 31) == 0) red[tid >> 5][i] = t;
    }
    __syncthreads();
    if (tid == 0) {
      double t[9];
      for (int i = 0; i < 9; ++i) t[i] = red[0][i] + red[1][i] + red[2][i] + red[3][i];
      const double m[3][3] = {{t[0], t[1], t[2]}, {t[1], t[3], t[4]}, {t[2], t[4], t[5]}};
      const double r[3] = {t[6], t[7], t[8]};
      const double det = det3(m);
      if (!(fabs(det) > 1e-12 * (m[0][0] * m[1][1] * m[2][2]))) {
        sol[3] = 0.0;
      } else {
        double x[3];
        for (int c = 0; c < 3; ++c) {
          double a[3][3];
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) a[i][j] = j == c ? r[i] : m[i][j];
          x[c] = det3(a) / det;
        }
        double nx = -x[1] / k, ny = -x[2] / k;
        double h2 = nx * nx + ny * ny;
        if (h2 > 1.0) {
          const double h = sqrt(h2);
          nx /= h;
          ny /= h;
          h2 = 1.0;
        }
        sol[0] = x[0];
        sol[1] = nx;
        sol[2] = ny;
        sol[3] = 1.0;
      }
    }
    __syncthreads();
    ok = sol[3] != 0.0;
    if (ok) nz = sqrt(1.0 - (sol[1] * sol[1] + sol[2] * sol[2]));
    __syncthreads();
  }
  if (!ok) {   // no direction: stop; the first fit failing marks the reconstruction failed
    if (tid == 0) {
      st->converged = 1;
      if (p.iteration == 0) {
        st->failed = 1;
        st->dir[0] = st->dir[1] = st->t0 = st->chi2 = __longlong_as_double(0x7ff8000000000000ll);
      } else {
        st->iterations = p.iteration;
      }
    }
    return;
  }
  const double nx = sol[1], ny = sol[2];
  const double zen = atan2(sqrt(nx * nx + ny * ny), nz);
  double az = atan2(ny, nx);
  if (az < 0.0) az += 2.0 * 3.14159265358979323846;
  // chi2 of this direction with these times (two-pass mean, as the per-direction residual)
  const double snx = sin(zen) * cos(az), sny = sin(zen) * sin(az), snz = cos(zen);
  double acc = 0.0;
  for (int s = tid; s < p.n_st; s += 128)
    acc += p.times[s] + (snx * p.pos[3 * s] + sny * p.pos[3 * s + 1] + snz * p.pos[3 * s + 2]) * k;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((tid & 31) == 0) red[tid >> 5][9] = acc;
  __syncthreads();
  const double mean = (red[0][9] + red[1][9] + red[2][9] + red[3][9]) / p.n_st;
  __syncthreads();
  double ss = 0.0;
  for (int s = tid; s < p.n_st; s += 128) {
    const double r = p.times[s] + (snx * p.pos[3 * s] + sny * p.pos[3 * s + 1] + snz * p.pos[3 * s + 2]) * k - mean;
    ss += r * r;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
  if ((tid & 31) == 0) red[tid >> 5][9] = ss;
  __syncthreads();
  if (tid == 0) {
    const double chi2 = red[0][9] + red[1][9] + red[2][9] + red[3][9];
    bool done = false;
    if (p.iteration > 0) {
      const double pz = st->dir[0], pa = st->dir[1];
      double dot = sin(pz) * cos(pa) * snx + sin(pz) * sin(pa) * sny + cos(pz) * snz;
      dot = dot > 1.0 ? 1.0 : (dot < -1.0 ? -1.0 : dot);
      done = same_s || acos(dot) < p.tol_rad;
      st->iterations = p.iteration;
    }
    st->dir[0] = zen;
    st->dir[1] = az;
    st->t0 = sol[0];
    st->chi2 = chi2;
    if (p.history) {
      p.history[2 * p.iteration] = zen;
      p.history[2 * p.iteration + 1] = az;
    }
    if (done) st->converged = 1;
  }
}

// the reconstruction's results into the caller's outputs
__global__ void recon_finish_kernel(const ReconState* st, double* direction, double* t0, double* chi2, int* iterations) {
  if (threadIdx.x != 0) return;
  direction[0] = st->dir[0];
  direction[1] = st->dir[1];
  *t0 = st->t0;
  *chi2 = st->chi2;
  *iterations = st->failed ? -1 : st->iterations;
}

}  // namespace aerafold
