// tc_dft.cuh -- the transforms of the unfolding as tensor-core DFTs (sm_103a, tcgen05).
//
// A precision variant of the FP32 FFT path (the forward transform of Sec. 4 and the inverse
// transform of the analytic signal, Sec. 2). Both transforms of an N-sample trace are split
// into 512-sample sub-blocks, A = N/512 of them. Only the M = N/4 bins of the 30-80 MHz band,
// k = k_lo + j (j < M), take part, and j = j1 + A j2 with j1 < A and j2 < M/A = 128:
//
//   forward   X[k_lo + j1 + A j2] = sum_n2 e^{-2 pi i j2 n2/512} W[j1][n2],
//             W[j1][n2] = e^{-2 pi i j1 n2/N} sum_n1 x'[512 n1 + n2] e^{-2 pi i j1 n1/A},
//             x'[n] = x[n] e^{-2 pi i k_lo n/N}
//   inverse   z[n2 + 512 n1] = e^{2 pi i k_lo n/N} sum_j1 e^{2 pi i j1 n1/A} e^{2 pi i j1 n2/N} Y[j1][n2],
//             Y[j1][n2] = sum_j2 Zf[k_lo + j1 + A j2] e^{2 pi i j2 n2/512}
//
// The 512 x 128 (forward) and 128 x 512 (inverse) complex DFT matrices are the GEMMs, one row
// per (station, channel, j1) or (pair, polarisation, j1). Complex numbers are stored as
// interleaved (re, im) pairs and the GEMMs are real: K = 1024, 256 output columns (forward)
// and K = 256, 1024 output columns (inverse). The A-point DFTs over the sub-block phase and
// the twiddles run in FP32 on the SIMT cores before (forward) and after (inverse) the GEMM.
//
// Precision: the GEMMs run on tensor cores in BF16 with FP32 accumulation. Each FP32 operand
// is split into BF16 parts (x = hi + mid + lo, each the round-to-nearest of what is left) and
// the products kept are those down to the target precision: 3 (hi*hi, hi*lo, lo*hi from a two-
// way split) or 6 (hi*hi, hi*mid, mid*hi, hi*lo, mid*mid, lo*hi from a three-way split). The
// DFT matrices are split on the host from FP64 values.
//
// Tensor-core details (PTX ISA, tcgen05). A persistent CTA (one per SM) computes 128 x 128
// tiles of D = A B^T (A row-major M x K, B row-major N x K, both K-major), each over a range
// of 64-wide K chunks, with 6 warps in three roles: warp 4 stages each chunk's operands with bulk copies into one of two
// shared-memory stages (mbarrier full/empty pairs), warp 5 issues the tcgen05.mma
// instructions (M 128, N 128, K 16; one per split product and K step) into tensor memory,
// and warps 0-3 read the chunk's partial sum out of tensor memory (tcgen05.ld) and fold it
// into the running sum (see the accumulation note below), writing the result at the end.
// Every wait is bounded. Operands come pre-split and pre-arranged in the shared-memory image
// of the no-swizzle K-major core-matrix layout: a core matrix is 8 rows x 16 bytes; in a
// 128-row, 64-column block the core matrix of rows 8a..8a+7 and columns 8b..8b+7 starts at
// byte 1024 a + 128 b (leading byte offset 128 along K, stride byte offset 1024 along M or N);
// one 16 KB block per (row tile, K chunk, plane), so a stage is filled by plain 1-D bulk
// copies. The producers of A (the forward pre-pass and the solve) write this image directly.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

#include "kernels.cuh"

namespace aerafold {
namespace tc {

constexpr int kSub = 512;                         // sub-block length
constexpr int kBandPhase = 128;                   // band bins per sub-block phase j1 (M / A)
constexpr int kBM = 128, kBN = 128, kBK = 64;     // CTA tile and K chunk
constexpr unsigned kErrBadLaunch = 2u;           // device error bit: a launch configuration the GEMM does not take
constexpr unsigned kBlk = kBM * kBK * 2;          // bytes of one BF16 plane of a 128 x 64 block (16 KB)
constexpr unsigned kStageBytes = 6 * kBlk;        // A and B, up to 3 planes each
constexpr int kStages = 2;                          // ring bytes: 2 such stages (x6) or 3 of 4 blocks (x3)
constexpr int kFwdK = 2 * kSub, kFwdN = 2 * kBandPhase;   // forward GEMM: K 1024, 256 outputs
constexpr int kInvK = 2 * kBandPhase, kInvN = 2 * kSub;   // inverse GEMM: K 256, 1024 outputs
constexpr size_t kEpiBytes = 4 * 32 * 32 * sizeof(float);   // a 32 x 32 transpose tile per fold warp
constexpr size_t kGemmSmem = kStages * kStageBytes + 256 + kEpiBytes;
constexpr int kGemmThreads = 192;

// byte offset of element (r, c) inside a 128-row, 64-column K-major BF16 block
__host__ __device__ constexpr unsigned core_offset(int r, int c) {
  return static_cast<unsigned>((r >> 3) * 1024 + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2);
}
// BF16 element offset of (row, k) in an image of rows x k (blocks [row / 128][k / 64])
__host__ __device__ constexpr size_t image_offset(int row, int k, int k_total) {
  return (static_cast<size_t>(row >> 7) * (k_total >> 6) + (k >> 6)) * (kBlk / 2) + core_offset(row & 127, k & 63) / 2;
}

// instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24
template <int BN>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(BN >> 3) << 17) | (uint32_t(kBM >> 4) << 24);
}

// shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading byte offset >> 4
// (bits 16-29), stride byte offset >> 4 (bits 32-45), version 1 (bits 46-47), no swizzle
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
  const uint64_t a = smem_u32(p);
  return ((a & 0x3FFFFull) >> 4) | (uint64_t(128 >> 4) << 16) | (uint64_t(1024 >> 4) << 32) | (1ull << 46);
}

// the products kept, as (plane of A, plane of B), most significant first
// (0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)
__host__ __device__ constexpr int term_a(int t) { return t == 2 || t == 4 ? 1 : t == 5 ? 2 : 0; }
__host__ __device__ constexpr int term_b(int t) { return t == 1 || t == 4 ? 1 : t == 3 ? 2 : 0; }

// The MMAs of one 64-wide K chunk held in the stage whose descriptor is base (A planes of
// 128 rows, then B planes of BN rows): for each 16-wide K step every kept product,
// accumulating into dst except at the first MMA of a fold unit. Unrolled with the terms
// fixed, so each MMA's descriptors are the base plus a constant.
template <int TERMS, int BN>
__device__ __forceinline__ void mma_chunk(uint64_t base, uint32_t dst, bool unit_first) {
  constexpr int planes = TERMS == 6 ? 3 : 2;
  constexpr uint32_t id = idesc<BN>();
#pragma unroll
  for (int ks = 0; ks < kBK / 16; ++ks) {
#pragma unroll
    for (int t = 0; t < TERMS; ++t) {
      const uint64_t ad = base + ((term_a(t) * kBlk + ks * 256) >> 4);
      const uint64_t bd = base + ((planes * kBlk + term_b(t) * (BN / 128) * kBlk + ks * 256) >> 4);
      const unsigned acc = (unit_first && ks == 0 && t == 0) ? 0u : 1u;
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dst),
          "l"(ad), "l"(bd), "r"(id), "r"(acc)
          : "memory");
    }
  }
}

struct GemmParams {
  const uint4* a[3];       // BF16 planes of A, image [m_tiles][chunks] of 16 KB blocks
  const uint4* b[3];       // BF16 planes of B, image [n_tiles][chunks] of 16 KB blocks
  float* d;                // D, row-major with row stride ldd; split-K group g at d + g * d_group
  size_t d_group;
  unsigned* err;
  int ldd, chunks, chunks_per_group, terms;   // terms 3 or 6
  int m_tiles, n_tiles, groups;               // work items: (m tile, n tile, K group), n fastest
};

// The work item of a persistent CTA's w-th item and the K chunks it covers.
struct GemmItem {
  int mt, nt, g;
};
__device__ __forceinline__ GemmItem gemm_item(const GemmParams& p, int w) {
  const int it = blockIdx.x + gridDim.x * w;
  GemmItem r;
  r.g = it % p.groups;
  r.nt = (it / p.groups) % p.n_tiles;
  r.mt = it / (p.groups * p.n_tiles);
  return r;
}

// FP32 -> BF16 parts, round to nearest at each step: x = hi + mid (+ lo)
__device__ __forceinline__ void split3(float x, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h);   // exact
  m = __float2bfloat16_rn(r1);
  l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// store complex value z at image element (row, 2 j) .. (row, 2 j + 1) of every plane
__device__ __forceinline__ void put_split(__nv_bfloat16* const (&img)[3], int planes, size_t off, float2 z) {
  __nv_bfloat16 h0, m0, l0, h1, m1, l1;
  split3(z.x, h0, m0, l0);
  split3(z.y, h1, m1, l1);
  *reinterpret_cast<__nv_bfloat162*>(img[0] + off) = __halves2bfloat162(h0, h1);
  *reinterpret_cast<__nv_bfloat162*>(img[1] + off) = __halves2bfloat162(m0, m1);
  if (planes == 3) *reinterpret_cast<__nv_bfloat162*>(img[2] + off) = __halves2bfloat162(l0, l1);
}

// 32 consecutive accumulator columns of this warp's 32 lanes: thread t gets row (32 w + t)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
      "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
      "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// arrives on the mbarrier once every tcgen05.mma this thread issued before it has completed
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Accumulation. The tensor cores' FP32 accumulator loses about 2^-26 of relative precision,
// with a bias, at every MMA (measured: the error grows linearly with the number of MMAs into
// one accumulator), so each fold unit (up to four 64-wide K chunks) is accumulated on its own
// into a partial region P[unit % 2] of tensor memory, and warps 0-3 fold it into the running
// sum S with IEEE round-to-nearest FP32 additions, in order: S = (((P0 + P1) + P2) + ...).
// With two partial regions the MMAs of one unit overlap the fold of the previous one.
// BN = 128: S, P0, P1 of 128 columns each; BN = 256 (x3 items of at most four chunks, which
// are single fold units and need no S): P0, P1 of 256 columns.
constexpr int kTmemCols = 512;

template <int BN>
__global__ void __launch_bounds__(kGemmThreads, 1) split_gemm_kernel(const __grid_constant__ GemmParams p) {
  static_assert(BN == 128 || BN == 256, "tile width");
  constexpr int NB = BN / 128;   // 128-row B blocks per tile
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* full = bars;          // [3] stage filled (bulk copies complete)
  uint64_t* empty = bars + 3;     // [3] stage consumed (its MMAs complete)
  uint64_t* ready = bars + 6;     // [2] partial region holds a finished chunk
  uint64_t* pfree = bars + 8;     // [2] partial region folded (4 arrivals, one per fold warp)
  uint64_t* done = bars + 10;     // every MMA complete
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(bars + 11);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int items = p.m_tiles * p.n_tiles * p.groups;
  // Persistent: this CTA takes items blockIdx.x, blockIdx.x + gridDim.x, ...; their chunks
  // form one stream (chunk i of the stream is chunk i % cpg of item i / cpg), so one item's
  // fold and store overlap the next item's copies and MMAs.
  const int my_items = blockIdx.x < items ? (items - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int cpg = p.chunks_per_group;
  const int nk = my_items * cpg;
  const int planes = p.terms == 6 ? 3 : 2;
  // The stage ring in the same 192 KB: three stages of 2 + 2 blocks (x3, BN 128), two of
  // 3 + 3 (x6, BN 128) or two of 2 + 4 (x3, BN 256).
  const unsigned stage_bytes = static_cast<unsigned>(planes * (1 + NB)) * kBlk;
  const int nst = min(3, static_cast<int>(kStages * kStageBytes / stage_bytes));
  // Chunks per fold: up to 4 (K = 256 accumulated on the tensor cores between folds), a
  // divisor of the item's chunk count; an item of at most 4 chunks is one fold unit, whose
  // fold only moves the accumulator to global memory.
  const int F = cpg <= 4 ? cpg : cpg % 4 == 0 ? 4 : cpg % 2 == 0 ? 2 : 1;
  const int nu = nk / F;   // fold units
  if (NB == 2 && (F != cpg || planes != 2)) {   // the wide tile has no running sum and room for 2 planes
    if (tid == 0) atomicOr(p.err, kErrBadLaunch);
    return;
  }

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(taddr_s)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int i = 0; i < 11; ++i) mbar_init(bars + i, (i == 8 || i == 9) ? 4 : 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t t_sum = *taddr_s;
  bool ok = true;

  if (warp == 4) {
    // ---- producer: bulk copies of each chunk's A and B blocks into a free stage ----
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < nk && ok; ++i) {
        const int s = i % nst;
        if (i >= nst) ok = mbar_wait_bounded(&empty[s], (i / nst - 1) & 1, kWaitLimitNs);
        if (!ok) break;
        const GemmItem w = gemm_item(p, i / cpg);
        const int kc = w.g * cpg + i % cpg;
        unsigned char* st = smem + s * stage_bytes;
        mbar_arrive_expect_tx(&full[s], stage_bytes);
        for (int pl = 0; pl < planes; ++pl) {
          tma_bulk_g2s(st + pl * kBlk, p.a[pl] + (static_cast<size_t>(w.mt) * p.chunks + kc) * (kBlk / 16), kBlk,
                       &full[s]);
          // the tile's NB consecutive 128-row B blocks: rows of the wider MMA continue in order
          for (int h = 0; h < NB; ++h)
            tma_bulk_g2s(st + (planes + pl * NB + h) * kBlk,
                         p.b[pl] + (static_cast<size_t>(w.nt * NB + h) * p.chunks + kc) * (kBlk / 16), kBlk, &full[s]);
        }
        issued = i + 1;
      }
      if (!ok) atomicOr(p.err, kErrTmaTimeout);
      // no copy may still be landing when the CTA leaves: wait (bounded) for the last ones
      for (int i = (issued > nst ? issued - nst : 0); i < issued; ++i)
        mbar_wait_bounded(&full[i % nst], (i / nst) & 1, kWaitLimitNs);
    }
  } else if (warp == 5) {
    // ---- MMA issuer ----
    if (lane == 0) {
      for (int i = 0; i < nk && ok; ++i) {
        const int s = i % nst;
        const int u = i / F, b = u & 1;              // fold unit and its partial region
        const bool unit_first = i % F == 0, unit_last = i % F == F - 1;
        ok = mbar_wait_bounded(&full[s], (i / nst) & 1, kWaitLimitNs);
        if (ok && unit_first && u >= 2) ok = mbar_wait_bounded(&pfree[b], ((u >> 1) - 1) & 1, kWaitLimitNs);
        if (!ok) break;
        tc_fence_after();
        const uint64_t base = smem_desc(smem + s * stage_bytes);
        const uint32_t dst = t_sum + (NB == 2 ? BN * b : BN * (1 + b));
        if (p.terms == 6) mma_chunk<6, BN>(base, dst, unit_first);
        else mma_chunk<3, BN>(base, dst, unit_first);
        tc_commit(&empty[s]);                  // the stage may be refilled
        if (unit_last) tc_commit(&ready[b]);   // the partial region may be folded
      }
      if (!ok) atomicOr(p.err, kErrTmaTimeout);
      tc_commit(done);
      mbar_wait_bounded(done, 0, kWaitLimitNs);   // no MMA outlives the tensor memory
    }
  } else {
    // ---- fold warps: S = S + P[chunk % 2]; an item's last chunk goes to global memory ----
    const uint32_t lanes = static_cast<uint32_t>(32 * warp) << 16;
    float4* epi = reinterpret_cast<float4*>(smem + kStages * kStageBytes + 256) + warp * 32 * 8;
    for (int u = 0; u < nu; ++u) {
      const int b = u & 1;
      ok = __all_sync(0xffffffffu, mbar_wait_bounded(&ready[b], (u >> 1) & 1, kWaitLimitNs));   // warp-uniform
      if (!ok) break;
      tc_fence_after();
      const int i = u * F;                  // the unit's first chunk
      const int kl = i % cpg;
      const bool first = kl == 0, last = kl + F == cpg;
      float* drow = nullptr;   // row 0 of the warp's 32 rows of the output tile
      if (last) {
        const GemmItem w = gemm_item(p, i / cpg);
        drow = p.d + w.g * p.d_group + static_cast<size_t>(w.mt * kBM + 32 * warp) * p.ldd + w.nt * BN;
      }
      const uint32_t preg = t_sum + (NB == 2 ? BN * b : BN * (1 + b));
#pragma unroll 1
      for (int c = 0; c < BN; c += 32) {
        uint32_t x[32], y[32];
        tmem_ld32(preg + lanes + c, x);
        if (!first) tmem_ld32(t_sum + lanes + c, y);
        tmem_wait_ld();
        if (!first) {
#pragma unroll
          for (int k = 0; k < 32; ++k) x[k] = __float_as_uint(__fadd_rn(__uint_as_float(y[k]), __uint_as_float(x[k])));
        }
        if (last) {
          // Lane l holds row l of the warp's 32 x 32 block. Transposed through shared memory
          // (16-byte chunk j of row r at chunk j ^ (r & 7): both sides free of bank conflicts)
          // so that each store instruction writes four rows of 128 contiguous bytes.
#pragma unroll
          for (int j = 0; j < 8; ++j)
            epi[lane * 8 + (j ^ (lane & 7))] = make_float4(__uint_as_float(x[4 * j]), __uint_as_float(x[4 * j + 1]),
                                                           __uint_as_float(x[4 * j + 2]), __uint_as_float(x[4 * j + 3]));
          __syncwarp();
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int r = 4 * i + (lane >> 3), ch = lane & 7;
            *reinterpret_cast<float4*>(drow + static_cast<size_t>(r) * p.ldd + c + 4 * ch) = epi[r * 8 + (ch ^ (r & 7))];
          }
          __syncwarp();   // the tile is read before the next block overwrites it
        } else {
          tmem_st32(t_sum + lanes + c, x);
        }
      }
      if (!last) tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&pfree[b]);
    }
    if (!ok && lane == 0) atomicOr(p.err, kErrTmaTimeout);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(t_sum), "r"(kTmemCols) : "memory");
  }
}

// Sum of the split-K groups' partial results, in group order (each group already folded its
// chunks in order): out[i] = ((part[0][i] + part[1][i]) + ...).
__global__ void tc_reduce_kernel(const float4* part, float4* out, size_t n4, size_t group4, int groups) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n4;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    float4 a = part[i];
    for (int gi = 1; gi < groups; ++gi) {
      const float4 b = part[gi * group4 + i];
      a = make_float4(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z), __fadd_rn(a.w, b.w));
    }
    out[i] = a;
  }
}

// ---- forward: phase rotation, A-point DFT over the sub-block phase, twiddle ----------------
// One CTA per (station, channel), thread n2; writes W[j1][n2] as GEMM row ((s * 2 + c) * A + j1),
// complex column n2, into the BF16 planes of the forward GEMM's A image.
struct SplitImage {
  __nv_bfloat16* plane[3];
  int planes;
};

template <int N_>
__global__ void __launch_bounds__(kSub) tc_forward_pre_kernel(const __grid_constant__ EventDesc ev,
                                                              const __grid_constant__ SplitImage img) {
  constexpr int N = N_, A = N / kSub;
  const int sc = blockIdx.x, n2 = threadIdx.x;
  const float* x = ev.traces + static_cast<size_t>(sc) * N;
  float2 y[A];
#pragma unroll
  for (int n1 = 0; n1 < A; ++n1) {
    const int n = n2 + kSub * n1;
    const float v = __ldg(x + n);
    const float2 ph = __ldg(ev.wn + ((ev.k_lo * n) & (N - 1)));   // exp(-2 pi i k_lo n / N)
    y[n1] = make_float2(v * ph.x, v * ph.y);
  }
  dft<A, -1>(y);
#pragma unroll
  for (int j1 = 0; j1 < A; ++j1) {
    const float2 t = j1 == 0 ? y[0] : cmul(y[j1], __ldg(ev.wn + j1 * n2));   // exp(-2 pi i j1 n2 / N)
    put_split(img.plane, img.planes, image_offset(sc * A + j1, 2 * n2, kFwdK), t);
  }
}

// ---- per pair: 2x2 solve (as the FP32 path) -> inverse GEMM rows --------------------------
// One CTA per pairs_per_cta consecutive pairs of the chunk [pair0, pair0 + n_pairs). Where the
// direction or the pattern changes, the CTA forms the scaled per-bin inverse of the VEL
// matrix in shared memory (build_inverse: corners read from the L2-resident table); each pair
// then applies it to its station's spectrum. The forward GEMM output holds X_c[k_lo + j1 + A j2]
// at row ((s * 2 + c) * A + j1), complex column j2. Zf goes to rows ((lp * 2 + pol) * A + j1),
// complex column j2, of the inverse GEMM's A image. Thread i takes column j2 = 4 (i / 4A) +
// i % 4 and row j1 = (i / 4) % A, so that a warp's stores fill whole 16-byte rows of the
// image's 8 x 8 core matrices (A rows of 16 bytes in a row for each polarisation).
constexpr int kSolvePairsMax = 32;   // pairs per solve CTA (consecutive: mostly one direction)
constexpr int kSolveThreads = 256;

template <int N_>
__global__ void __launch_bounds__(kSolveThreads) tc_solve_kernel(const __grid_constant__ EventDesc ev,
                                                                 const float2* xf,
                                                                 const __grid_constant__ SplitImage img,
                                                                 long long pair0, int n_pairs, int pairs_per_cta) {
  constexpr int N = N_, M = N / 4, A = N / kSub, T = kSolveThreads;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* hinv = reinterpret_cast<float4*>(smem_raw);                         // [2][M]
  float2* hn = reinterpret_cast<float2*>(smem_raw + 2 * sizeof(float4) * M);  // [n_f][8]
  __shared__ DirInfo s_di;
  const int tid = threadIdx.x;
  const int S = ev.n_st;
  int cur_d = -1, cur_p = -3;
  DirInfo di;
  bool key_sing = false;
  for (int k = 0; k < pairs_per_cta; ++k) {
    const int lp = blockIdx.x * pairs_per_cta + k;   // pair within the chunk
    if (lp >= n_pairs) break;
    const long long pair = pair0 + lp;
    const int d = static_cast<int>(pair / S), s = static_cast<int>(pair % S);
    const int p = station_pattern(ev, s);
    if (d != cur_d || p != cur_p) {
      // new direction or pattern: the cell (FP64) by one thread (FP64 is a small fraction of
      // the FP32 rate), then the per-bin inverse
      __syncthreads();   // the previous pair's reads of hinv are done
      if (tid == 0) s_di = pair_cell(ev, d, p, nullptr);
      __syncthreads();
      di = s_di;
      key_sing = build_inverse<N_, T>(ev, p, di, nullptr, true, hn, hinv);
      cur_d = d;
      cur_p = p;
    }
    const float2* x0 = xf + static_cast<size_t>(s * 2) * A * kBandPhase;
    const float2* x1 = x0 + A * kBandPhase;
#pragma unroll
    for (int it = 0; it < M / T; ++it) {
      const int i = tid + T * it;
      const int j1 = (i / 4) % A, j2 = 4 * (i / (4 * A)) + i % 4;
      const int j = j1 + A * j2;
      const float4 h0 = hinv[j], h1 = hinv[M + j];   // (h00, h01), (h10, h11)
      const float2 v0 = x0[j1 * kBandPhase + j2], v1 = x1[j1 * kBandPhase + j2];
      float2 et, ep;
      et.x = fmaf(h0.z, v1.x, fmaf(-h0.w, v1.y, fmaf(h0.x, v0.x, -h0.y * v0.y)));
      et.y = fmaf(h0.z, v1.y, fmaf(h0.w, v1.x, fmaf(h0.x, v0.y, h0.y * v0.x)));
      ep.x = fmaf(h1.z, v1.x, fmaf(-h1.w, v1.y, fmaf(h1.x, v0.x, -h1.y * v0.y)));
      ep.y = fmaf(h1.z, v1.y, fmaf(h1.w, v1.x, fmaf(h1.x, v0.y, h1.y * v0.x)));
      put_split(img.plane, img.planes, image_offset((lp * 2) * A + j1, 2 * j2, kInvK), et);
      put_split(img.plane, img.planes, image_offset((lp * 2 + 1) * A + j1, 2 * j2, kInvK), ep);
    }
    if (tid == 0) ev.status[pair] = di.st | (key_sing ? kStSingular : 0u);
  }
}

// ---- inverse: twiddle, A-point DFT over the sub-block phase, band phase, envelope, peak ----
// One CTA per pair of the chunk, thread n2; the inverse GEMM output holds Y[j1][n2] at row
// ((lp * 2 + pol) * A + j1), complex column n2.
template <int N_>
__global__ void __launch_bounds__(kSub) tc_inverse_post_kernel(const __grid_constant__ EventDesc ev,
                                                               const float2* y_in, long long pair0) {
  constexpr int N = N_, A = N / kSub;
  const int lp = blockIdx.x, n2 = threadIdx.x;
  const long long pair = pair0 + lp;
  const int s = static_cast<int>(pair % ev.n_st);
  float pw[A];
#pragma unroll
  for (int i = 0; i < A; ++i) pw[i] = 0.f;
#pragma unroll
  for (int pol = 0; pol < 2; ++pol) {
    float2 y[A];
    const float2* rows = y_in + static_cast<size_t>(lp * 2 + pol) * A * kSub;
#pragma unroll
    for (int j1 = 0; j1 < A; ++j1) {
      const float2 v = rows[j1 * kSub + n2];
      y[j1] = j1 == 0 ? v : cmulc(v, __ldg(ev.wn + j1 * n2));   // exp(+2 pi i j1 n2 / N)
    }
    dft<A, +1>(y);
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) {
      const int n = n2 + kSub * n1;
      const float2 zz = cmulc(y[n1], __ldg(ev.wn + ((ev.k_lo * n) & (N - 1))));   // exp(+2 pi i k_lo n / N)
      if (ev.efield) ev.efield[(static_cast<size_t>(pair) * 2 + pol) * N + n] = zz.x;
      pw[n1] += cabs2(zz);
    }
  }
  __shared__ float senv[N];   // for the sub-sample peak
  float bv = -1.f;
  int bi = 0;
#pragma unroll
  for (int n1 = 0; n1 < A; ++n1) {
    const int n = n2 + kSub * n1;
    const float v = sqrtf(pw[n1]);
    if (ev.envelope) ev.envelope[static_cast<size_t>(pair) * N + n] = v;
    senv[n] = v;
    if (v > bv) { bv = v; bi = n; }
  }
  __shared__ float rv[kSub / 32];
  __shared__ int ri[kSub / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, bv, off);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
  }
  if ((n2 & 31) == 0) { rv[n2 >> 5] = bv; ri[n2 >> 5] = bi; }
  __syncthreads();
  __shared__ float pk_v;
  __shared__ int pk_i;
  if (n2 == 0) {
    for (int w = 1; w < kSub / 32; ++w)
      if (rv[w] > bv || (rv[w] == bv && ri[w] < bi)) { bv = rv[w]; bi = ri[w]; }
    if (bv < 0.f) { bv = 0.f; bi = 0; }
    pk_v = bv;
    pk_i = bi;
    ev.peak_idx[pair] = bi;
    ev.peak_amp[pair] = bv;   // the peak time is formed with the direction's residual
    if (ev.peak_fine)
      ev.peak_fine[pair] =
          __dadd_rn(ev.t_start[s], __dmul_rn(__dadd_rn(static_cast<double>(bi), peak_offset(senv, N, bi)), ev.dt_ns));
  }
  if (ev.snr) {
    __shared__ float rw[kSub / 32];
    __syncthreads();   // the pair's peak visible to every thread
    const float snr = pair_snr<kSub>(senv, N, pk_i, pk_v, rw);
    if (n2 == 0) ev.snr[pair] = snr;
  }
}

// ---- per direction: the FP64 plane-wave timing residual ------------------------------------
__global__ void __launch_bounds__(128) tc_residual_kernel(const __grid_constant__ EventDesc ev) {
  __shared__ double red[128 / 32];
  direction_residual<128>(ev, blockIdx.x, red);
}

}  // namespace tc
}  // namespace aerafold
