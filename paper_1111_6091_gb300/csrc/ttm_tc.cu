// n-mode products Y = Z x_n R-hat on tcgen05 tensor cores (Eq. ctensor_transformed).
//
// Each mode product is a GEMM whose tensor-core M dimension is a large index of Z and whose
// N dimension is the coarse size Ic (<= 256), with L = prod_{m<n} I_m, G = prod_{m>n} I_m:
//   n = 1 : Y(c, g)    = sum_k R-hat(c, k) Z(k, g)     D(g, c), A(g, k) = Z(k, g)
//   n > 1 : Y(l, c, g) = sum_k Z(l, k, g) R-hat(c, k)  D(l, c), A(l, k) = Z(l, k, g), per g
// B is R-hat with c contiguous (MN-major) in shared memory.
//
// Precision (split BF16): every float x is hi + lo with hi = bf16(x), lo = bf16(x - hi).  The
// products hi*hi + hi*lo + lo*hi are accumulated in FP32 in tensor memory; the dropped lo*lo
// term and the rounding of lo leave a relative error near 2^-16 per product.
//
// The A operand lives in tensor memory. Splitter threads own one row of the 128-row tile each
// (its tensor-memory lane). A thread splits the 16 k values of a half-step and writes hi and lo
// with tcgen05.st. The MMA reads A from there and only B from shared memory. Shared memory carries
// the fp32 tiles of Z, written by TMA and read once by the splitters, and a ring of pre-split R-hat
// chunks.
//
// Persistent CTAs of 736 threads, one per SM, walk 128-row output tiles:
//   warp 0      producer: fp32 tiles of Z by cp.async.bulk.tensor (128-byte swizzle)
//   warp 1      producer: pre-split R-hat chunks through a 2-D tensor map (bulk copies if that
//               cannot be encoded), one slot per K step in flight
//   warp 2      allocates tensor memory. One lane issues a K step at a time: six tcgen05.mma
//               (hi*hi + hi*lo + lo*hi for two K16 halves, A from tensor memory), then one commit
//               that frees the step's R-hat slot and A stage pair. The same instruction block
//               tests the next step's barriers without blocking, so those waits overlap the MMAs.
//   warps 3-18  splitters: four groups of four warps (one per lane quarter) take the K16
//               half-steps in turn, so four are in flight at once. When Z's strides do not
//               suit a tensor map, they load Z straight from global memory.
//   warps 19-22 drain an accumulator while the next tile is computed. There are two
//               accumulators, at columns 0 and 256, when Ic <= 208, else one. Mode-1 tiles
//               leave through TMA stores from a swizzled staging buffer.
// Every mbarrier wait gives up after about 2 s, records an error and lets the CTA unwind.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "ttm.cuh"

namespace cpmg {

namespace {

constexpr int BMT = 128;                       // tensor-core M tile (TMEM lanes)
constexpr int BKT = 32;                        // K per pipeline stage (two MMA K steps)
constexpr int kZWarp = 0;                      // fp32 Z tile producer
constexpr int kBWarp = 1;                      // R-hat chunk producer
constexpr int kMmaWarp = 2;                    // tensor-memory owner and MMA issuer
constexpr int kSplitWarp0 = 3;                 // splitter warps: kGroups groups of four
constexpr int kGroups = 4;
constexpr int kSplitWarps = 4 * kGroups;
constexpr int kEpiWarp0 = kSplitWarp0 + kSplitWarps;  // four epilogue warps
constexpr int THREADS = 32 * (kEpiWarp0 + 4);
constexpr int kTmemCols = 512;                 // the whole of an SM's tensor memory
constexpr int kAccStride = 256;                // second accumulator's first column
constexpr int kAStageCols = 16;                // per K16 half-step: hi (8 columns), lo (8 columns)
constexpr int kMaxAStages = 8;
constexpr int kMaxRing = 8;
constexpr uint32_t kF32Bytes = BMT * BKT * 4;  // fp32 staging of one stage
constexpr int kStageBase = 1024;               // 128-byte swizzle wants 1 KB alignment

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool bar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}


__device__ __forceinline__ bool failed(const int* fail) { return *reinterpret_cast<const volatile int*>(fail) != 0; }

// bounded wait: false after ~2 s without the phase completing, or once another role of the
// CTA has recorded a failure in *fail (fail null: only the phase or the time limit ends it)
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, const int* fail) {
  if (bar_try(bar, parity)) return true;
  const uint64_t t0 = gtime();
  while (true) {
    if (bar_try(bar, parity)) return true;
    if ((fail && failed(fail)) || gtime() - t0 > 2000000000ull) return false;
  }
}

// the same for a whole warp: lane 0 polls the barrier (32 lanes polling one mbarrier would
// queue 32 shared-memory operations per test), then the warp synchronizes, which orders the
// other lanes' later reads after lane 0's observation of the phase
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, const int* fail) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = bar_wait(bar, parity, fail) ? 1 : 0;
  __syncwarp();
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// cursor over a ring of S slots: the slot, and the parity of the phase its current use
// completes (no divisions in the loops)
struct Ring {
  int slot, S;
  uint32_t phase;
  __device__ explicit Ring(int s) : slot(0), S(s), phase(0) {}
  __device__ void next() {
    if (++slot == S) {
      slot = 0;
      phase ^= 1u;
    }
  }
};

__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void bar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(su32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

// shared-memory matrix descriptor: start, leading / stride byte offsets, tcgen05 version,
// no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// One 32-wide K step of split BF16 (two K16 half-steps, six MMAs), then a commit that arrives
// on `done` once they have completed.  The block first tests (without blocking) phase p0 of
// barrier b0 and phase p1 of b1, so that the latency of the tests overlaps the MMA issue; bit 0
// / bit 1 of the result report them.
__device__ __forceinline__ uint32_t mma6_commit_test(uint32_t d, uint32_t a0h, uint32_t a0l, uint32_t a1h, uint32_t a1l,
                                                     uint64_t b0h, uint64_t b0l, uint64_t b1h, uint64_t b1l,
                                                     uint32_t idesc, uint32_t acc, const uint64_t* done,
                                                     const uint64_t* t0, uint32_t p0, const uint64_t* t1, uint32_t p1) {
  uint32_t r0, r1;
  asm volatile(
      "{\n\t.reg .pred pa, pt, q0, q1;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 q0, [%14], %15;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 q1, [%16], %17;\n\t"
      "setp.ne.b32 pa, %12, 0;\n\t"
      "setp.eq.b32 pt, %12, %12;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%2], [%3], %7, %11, pa;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%2], [%3], %8, %11, pt;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%2], [%4], %7, %11, pt;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%2], [%5], %9, %11, pt;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%2], [%5], %10, %11, pt;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%2], [%6], %9, %11, pt;\n\t"
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%13];\n\t"
      "selp.u32 %0, 1, 0, q0;\n\t"
      "selp.u32 %1, 1, 0, q1;\n\t}"
      : "=r"(r0), "=r"(r1)
      : "r"(d), "r"(a0h), "r"(a0l), "r"(a1h), "r"(a1l), "l"(b0h), "l"(b0l), "l"(b1h), "l"(b1l), "r"(idesc),
        "r"(acc), "r"(su32(done)), "r"(su32(t0)), "r"(p0), "r"(su32(t1)), "r"(p1)
      : "memory");
  return r0 | (r1 << 1);
}

// eight 32-bit columns of this warp's 32 tensor-memory lanes (lane i of the warp writes lane
// base + i)
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}

// sixteen 32-bit columns of this warp's 32 tensor-memory lanes (completion: tcgen05.wait::ld)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// x -> (hi, lo) for 16 floats; column j packs elements 2j (low half) and 2j + 1 (high half),
// the order of consecutive K elements in memory.  Two floats per conversion instruction; a
// BF16 value widens to float exactly by a 16-bit shift.
__device__ __forceinline__ void split16(const float* x, uint32_t* hi, uint32_t* lo) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
    const uint32_t hb = *reinterpret_cast<const uint32_t*>(&h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x[2 * j] - __uint_as_float(hb << 16),
                                                   x[2 * j + 1] - __uint_as_float(hb & 0xffff0000u));
    hi[j] = hb;
    lo[j] = *reinterpret_cast<const uint32_t*>(&l);
  }
}

// byte offset of 16-byte chunk `chunk` of 128-byte row `row` under the 128-byte swizzle
__device__ __forceinline__ uint32_t sw128(int row, int chunk) {
  return (uint32_t)row * 128u + (uint32_t)((chunk ^ (row & 7)) << 4);
}

struct TcArgs {
  int first;            // 1: mode 1 (rows of A are g, k contiguous), 0: later mode (rows are l)
  int direct;           // 1: splitters load Z from global memory (no tensor map)
  int btm;              // 1: R-hat chunks through their tensor map (rows of 128 bytes), else bulk copies
  int ytm;              // 1: mode-1 output tiles through TMA stores (Y rows of Ic floats)
  int sf, sb, sa;       // slots of the fp32 ring, of the R-hat ring, K16 A stages in tensor memory
  int nacc;             // accumulators in tensor memory: 1 (at column 0) or 2 (at 0 and 256)
  int n0;               // A stages after the first accumulator; the rest follow the second
  int64_t M, K, Ic;     // GEMM sizes: spatial rows, contracted index, coarse size
  int Npad;             // Ic rounded up to a multiple of 16
  int64_t batch;        // G for a later mode, 1 for mode 1
  int64_t mtiles;
  int64_t ntiles;       // mtiles * batch
  const float* Z;
  const unsigned char* bsplit;  // pre-split R-hat: per K chunk [hi | lo], canonical MN-major
  uint32_t bchunk;      // bytes of one BF16 term of one R-hat chunk (Npad * BKT * 2)
  float* Y;
  int64_t ldy_m, ldy_c, ldy_b;
  int vec4;             // Y rows hold Ic contiguous floats, 16-byte aligned: float4 stores
  int* err;
};


// Persistent: CTA b handles tiles b, b + gridDim.x, ...  Three rings: fp32 tiles of Z in shared
// memory (freed as soon as they are split, so Z loads run several stages ahead), R-hat chunks
// in shared memory and A stages in tensor memory (both freed by the MMA commit).  With two
// accumulators the epilogue of one tile overlaps the main loop of the next.
__global__ void __launch_bounds__(THREADS, 1) k_ttm_tc(const __grid_constant__ CUtensorMap tmap,
                                                        const __grid_constant__ CUtensorMap bmap,
                                                        const __grid_constant__ CUtensorMap ymap, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int SF = a.sf, SB = a.sb, NA = a.nacc;  // A stages: 2 SB (a pair per K step)
  // first tensor-memory column of K16 A stage s: the columns after each accumulator
  auto stage_col = [&](int s) -> uint32_t {
    return (uint32_t)(s < a.n0 ? a.Npad + kAStageCols * s : kAccStride + a.Npad + kAStageCols * (s - a.n0));
  };
  uint64_t* ffull = reinterpret_cast<uint64_t*>(smem);  // fp32 tile landed
  uint64_t* fempty = ffull + kMaxRing;                  // fp32 tile read by the splitters
  uint64_t* bfull = fempty + kMaxRing;                  // R-hat chunk landed
  uint64_t* kempty = bfull + kMaxRing;                  // MMAs of a K step completed: its R-hat
                                                        // slot and A stage pair are free
  uint64_t* afull = kempty + kMaxRing;                  // A stage written to tensor memory
  uint64_t* tfull = afull + kMaxAStages;                // [2] accumulator complete
  uint64_t* tempty = tfull + 2;                         // [2] accumulator drained
  uint64_t* mdone = tempty + 2;                         // every MMA issued has completed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 512);
  int* fail = reinterpret_cast<int*>(smem + 520);
  unsigned char* fring = smem + kStageBase;
  unsigned char* bring = fring + (size_t)SF * kF32Bytes;
  // TMA-store staging: per epilogue warp two 4 KB buffers (32 rows x 128 bytes, 128-byte swizzle)
  unsigned char* ystage = smem + (((uint32_t)(bring - smem) + (uint32_t)SB * 2u * a.bchunk + 1023u) & ~1023u);
  const uint32_t bslot = 2 * a.bchunk;
  const int nk = (int)((a.K + BKT - 1) / BKT);
  // CTAs start their K loops at different chunks, so that the SMs do not all read the same
  // R-hat chunk at the same moment
  const int rot = (int)(blockIdx.x % nk);
  const uint32_t b_lbo = (uint32_t)(a.Npad / 8) * 128u, b_sbo = 128u;

  if (t == 0) {
    for (int s = 0; s < kMaxRing; ++s) {
      bar_init(&ffull[s], 1);
      bar_init(&fempty[s], 8);  // the two half-steps of a stage, four warps each
      bar_init(&bfull[s], 1);
      bar_init(&kempty[s], 1);
    }
    for (int s = 0; s < kMaxAStages; ++s) bar_init(&afull[s], 8);  // both half-steps, four warps each
    for (int j = 0; j < 2; ++j) {
      bar_init(&tfull[j], 1);
      bar_init(&tempty[j], 4);
    }
    bar_init(mdone, 1);
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (warp == kZWarp || warp == kBWarp) {
    // ------------------------------------------------------------ producers
    const bool zp = warp == kZWarp;
    if (lane == 0 && !(zp && a.direct)) {
      const int S = zp ? SF : SB;
      uint64_t* fullb = zp ? ffull : bfull;
      uint64_t* emptyb = zp ? fempty : kempty;
      Ring r(S);
      int it = 0, kq = rot;
      for (int64_t tile = blockIdx.x; tile < a.ntiles && !failed(fail); tile += gridDim.x) {
        const int64_t b = tile / a.mtiles;
        const int m0 = (int)((tile % a.mtiles) * BMT);
        for (int kc = 0; kc < nk; ++kc, ++it) {
          if (it >= S && !bar_wait(&emptyb[r.slot], r.phase ^ 1u, fail)) {
            atomicOr(fail, 1);
            break;
          }
          const int k0 = kq * BKT;
          if (zp) {
            unsigned char* st = fring + (size_t)r.slot * kF32Bytes;
            bar_arrive_tx(&fullb[r.slot], kF32Bytes);
            if (a.first) {
              // box {BKT along k, BMT along g}: 128 rows of 128 bytes
              asm volatile(
                  "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                  "[%4];" ::"r"(su32(st)),
                  "l"(&tmap), "r"(k0), "r"(m0), "r"(su32(&fullb[r.slot]))
                  : "memory");
            } else {
              // four boxes {32 along l, BKT along k, 1}: each 32 rows (k) of 128 bytes (l)
              for (int q = 0; q < BMT / 32; ++q)
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                    "%4}], [%5];" ::"r"(su32(st + q * 4096)),
                    "l"(&tmap), "r"(m0 + 32 * q), "r"(k0), "r"((int)b), "r"(su32(&fullb[r.slot]))
                    : "memory");
            }
          } else {
            unsigned char* st = bring + (size_t)r.slot * bslot;
            bar_arrive_tx(&fullb[r.slot], bslot);
            if (a.btm) {
              // box {64 BF16, Npad rows}: the chunk's Npad rows of 128 bytes, in order
              asm volatile(
                  "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                  "[%4];" ::"r"(su32(st)),
                  "l"(&bmap), "r"(0), "r"(kq * a.Npad), "r"(su32(&fullb[r.slot]))
                  : "memory");
            } else {
              const unsigned char* src = a.bsplit + (size_t)kq * bslot;
              asm volatile(
                  "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                      su32(st)),
                  "l"(src), "r"(bslot), "r"(su32(&fullb[r.slot]))
                  : "memory");
            }
          }
          r.next();
          if (++kq == nk) kq = 0;
        }
      }
      // the CTA may not exit while a copy is still in flight (this wait ignores the failure
      // flag: only the copy's own completion, or the time limit, ends it)
      for (int j = (it > S ? it - S : 0); j < it; ++j)
        if (!bar_wait(&fullb[j % S], (uint32_t)((j / S) & 1), nullptr)) atomicOr(fail, 1);
    }
  } else if (warp >= kSplitWarp0 && warp < kEpiWarp0) {
    // ------------------------------------------------------------ split fp32 -> BF16 hi / lo
    // Half-step hs = 2 it + h covers k = 16 h .. 16 h + 15 of K step `it`.  Group g (four
    // warps, one per lane quarter) takes half-steps g, g + kGroups, ..., so that kGroups
    // half-steps are in flight at once.  A thread owns row 32 q + lane of the tile (its
    // tensor-memory lane); hi goes to the 8 columns of its A stage, lo to the next 8.
    const int q = warp & 3, g = (warp - kSplitWarp0) >> 2;
    const int r = 32 * q + lane;
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    // cursors for half-step hs: K step it = hs / 2 (tile tile_i = it / nk, chunk kc = it % nk),
    // fp32 slot it % SF, A stage pair it % SB (stage 2 pair + h)
    int hs = g, it = g >> 1, kc = it, kq = 0;
    int64_t tile = blockIdx.x;
    while (kc >= nk) {
      kc -= nk;
      tile += gridDim.x;
    }
    kq = kc + rot;
    if (kq >= nk) kq -= nk;
    int fslot = 0, pslot = it % SB;
    uint32_t fph = 0, pph = (uint32_t)((it / SB) & 1);
    if (SF > 0) {
      fslot = it % SF;
      fph = (uint32_t)((it / SF) & 1);
    }
    while (tile < a.ntiles) {
      const int h = hs & 1;
      const int64_t b = tile / a.mtiles;
      const int64_t m = (tile % a.mtiles) * BMT + r;
      const int64_t k0 = (int64_t)kq * BKT + 16 * h;
      float x[16];
      if (a.direct) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int64_t k = k0 + i;
          x[i] = (m < a.M && k < a.K) ? __ldg(a.first ? a.Z + k + a.K * m : a.Z + m + a.M * k + a.M * a.K * b) : 0.f;
        }
      } else {
        if (!warp_wait(&ffull[fslot], fph, fail)) {
          if (lane == 0) atomicOr(fail, 1);
          break;
        }
        const unsigned char* st = fring + (size_t)fslot * kF32Bytes;
        if (a.first) {
          // row r: 128 bytes under the 128-byte swizzle; this half is chunks 4 h .. 4 h + 3
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 v = *reinterpret_cast<const float4*>(st + sw128(r, 4 * h + j));
            x[4 * j] = v.x; x[4 * j + 1] = v.y; x[4 * j + 2] = v.z; x[4 * j + 3] = v.w;
          }
        } else {
          // box q holds rows k (128 bytes of l each); this lane's l is float `lane` of a row
          const unsigned char* box = st + q * 4096 + (lane & 3) * 4;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int kk = 16 * h + i;
            x[i] = *reinterpret_cast<const float*>(box + kk * 128 + (((lane >> 2) ^ (kk & 7)) << 4));
          }
        }
      }
      uint32_t hi[8], lo[8];
      split16(x, hi, lo);
      if (!a.direct) {
        __syncwarp();
        if (lane == 0) bar_arrive(&fempty[fslot]);
      }
      // the A stage pair is free once the MMAs of its previous K step have completed
      if (it >= SB && !warp_wait(&kempty[pslot], pph ^ 1u, fail)) {
        if (lane == 0) atomicOr(fail, 1);
        break;
      }
      const int aslot = 2 * pslot + h;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t col = tmem + lanes + stage_col(aslot);
      tmem_st8(col, hi);
      tmem_st8(col + 8, lo);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) bar_arrive(&afull[pslot]);
      // advance by kGroups half-steps
      const int nit = (hs + kGroups) >> 1, dit = nit - it;
      hs += kGroups;
      it = nit;
      kc += dit;
      kq += dit;
      while (kq >= nk) kq -= nk;
      while (kc >= nk) {
        kc -= nk;
        tile += gridDim.x;
      }
      if (SF > 0) {
        fslot += dit;
        while (fslot >= SF) {
          fslot -= SF;
          fph ^= 1u;
        }
      }
      pslot += dit;
      while (pslot >= SB) {
        pslot -= SB;
        pph ^= 1u;
      }
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      // D F32, A and B BF16, A K-major (rows in tensor-memory lanes), B MN-major, N = Npad,
      // M = 128
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((uint32_t)(a.Npad >> 3) << 17) |
                             ((uint32_t)(BMT >> 4) << 24);
      Ring rp(SB), rt(NA);
      const uint64_t dB0 = sdesc(su32(bring), b_lbo, b_sbo);
      int i = 0;
      bool ok = true;
      // a_ok / b_ok: the next A stage / R-hat chunk was seen complete by the test issued
      // alongside the previous MMAs, so its blocking wait is skipped
      bool a_ok = false, b_ok = false;
      for (int64_t tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x, ++i) {
        if (i >= NA && !bar_wait(&tempty[rt.slot], rt.phase ^ 1u, fail)) {
          atomicOr(fail, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(rt.slot * kAccStride);
        for (int kc = 0; kc < nk && ok; ++kc) {
          if (!b_ok && !bar_wait(&bfull[rp.slot], rp.phase, fail)) {
            atomicOr(fail, 1);
            ok = false;
            break;
          }
          // a descriptor's start-address field is the shared-memory address / 16 (below 2^18
          // bytes, so the field never carries): slot, half-step and hi / lo are added offsets
          const uint64_t dBh = dB0 + ((uint32_t)rp.slot * bslot >> 4), dBl = dBh + (a.bchunk >> 4);
          Ring np = rp;
          np.next();
          if (!a_ok && !bar_wait(&afull[rp.slot], rp.phase, fail)) {
            atomicOr(fail, 1);
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          // both half-steps, the commit that frees the K step's R-hat slot and A stage pair, and
          // tests of the next K step's A stage pair and R-hat chunk
          static_assert(BKT == 32, "one K step is two K16 half-steps");
          const uint32_t a0 = tmem + stage_col(2 * rp.slot), a1 = tmem + stage_col(2 * rp.slot + 1);
          const uint64_t bo = (2 * b_lbo) >> 4;
          const uint32_t seen = mma6_commit_test(d, a0, a0 + 8, a1, a1 + 8, dBh, dBl, dBh + bo, dBl + bo, idesc,
                                                 kc > 0 ? 1u : 0u, &kempty[rp.slot], &afull[np.slot], np.phase,
                                                 &bfull[np.slot], np.phase);
          a_ok = (seen & 1u) != 0;
          b_ok = (seen & 2u) != 0;
          rp = np;
        }
        // accumulator `rt.slot` is complete once every MMA issued so far has finished
        if (ok) mma_commit(&tfull[rt.slot]);
        rt.next();
      }
      // tensor memory is released only after every MMA issued has completed
      mma_commit(mdone);
      if (!bar_wait(mdone, 0, nullptr)) atomicOr(fail, 1);
    }
  } else {
    // ------------------------------------------------------------ epilogue (4 warps): TMEM -> Y
    const int quarter = warp & 3;  // a warp reaches TMEM lanes 32 * (warp id mod 4) .. + 31
    Ring rt(NA);
    unsigned char* stg = ystage + quarter * 8192;
    int nst = 0;  // TMA stores this warp has issued (their buffer alternates)
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
      if (!warp_wait(&tfull[rt.slot], rt.phase, fail)) {
        if (lane == 0) atomicOr(fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int64_t b = tile / a.mtiles;
      const int64_t row0 = (tile % a.mtiles) * BMT + 32 * quarter;
      const int64_t row = row0 + lane;
      const uint32_t base = tmem + (uint32_t)(rt.slot * kAccStride) + ((uint32_t)(32 * quarter) << 16);
      if (a.ytm) {
        // 32 columns at a time: TMEM -> registers -> swizzled staging -> one TMA store of a
        // 32 x 32 box (rows past M and columns past Ic are clipped by the copy)
        for (int c0 = 0; c0 < a.Npad; c0 += 32, ++nst) {
          uint32_t v[32];
          tmem_ld16(base + (uint32_t)c0, v);
          if (c0 + 16 < a.Npad) {
            tmem_ld16(base + (uint32_t)(c0 + 16), v + 16);
          } else {
#pragma unroll
            for (int j = 16; j < 32; ++j) v[j] = 0u;
          }
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          unsigned char* buf = stg + (nst & 1) * 4096;
          // the buffer's previous store (two stores ago) must have read it
          if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
          __syncwarp();
#pragma unroll
          for (int j = 0; j < 8; ++j)
            *reinterpret_cast<uint4*>(buf + sw128(lane, j)) = make_uint4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) {
            asm volatile(
                "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(&ymap), "r"(c0),
                "r"((int)row0), "r"(su32(buf))
                : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          }
        }
      } else {
        float* y = a.Y + b * a.ldy_b + row * a.ldy_m;
        for (int c0 = 0; c0 < a.Npad; c0 += 16) {
          uint32_t v[16];
          tmem_ld16(base + (uint32_t)c0, v);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (row < a.M) {
            if (a.vec4) {
#pragma unroll
              for (int j = 0; j < 16; j += 4)
                if (c0 + j < a.Ic)
                  *reinterpret_cast<float4*>(y + c0 + j) =
                      make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]), __uint_as_float(v[j + 2]),
                                  __uint_as_float(v[j + 3]));
            } else {
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if (c0 + j < a.Ic) y[(int64_t)(c0 + j) * a.ldy_c] = __uint_as_float(v[j]);
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) bar_arrive(&tempty[rt.slot]);
      rt.next();
    }
    // the CTA may not exit (and its shared memory be reused) before its stores have read it
    if (a.ytm && lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  if (t == 0 && *fail && a.err) atomicOr(a.err, 1);
}

// R-hat (Ic x In, float64, column-major) -> per K chunk of BKT: [hi | lo] BF16 in the canonical
// MN-major layout (c fastest within a core-matrix row), zero beyond Ic or In.
__global__ void k_split_rhat(const double* Rh, int64_t Ic, int64_t In, int Npad, int nk, uint32_t bchunk,
                             unsigned char* out) {
  const uint32_t lbo = (uint32_t)(Npad / 8) * 128u;
  const int64_t total = (int64_t)nk * Npad * BKT;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / ((int64_t)Npad * BKT);
    const int rem = (int)(e % ((int64_t)Npad * BKT));
    const int c = rem % Npad, kk = rem / Npad;
    const int64_t k = q * BKT + kk;
    const float x = (c < Ic && k < In) ? (float)Rh[c + Ic * k] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    unsigned char* base = out + (size_t)q * 2 * bchunk;
    const uint32_t o = (uint32_t)(c >> 3) * 128u + (uint32_t)(kk >> 3) * lbo + (uint32_t)(kk & 7) * 16u +
                       (uint32_t)(c & 7) * 2u;
    *reinterpret_cast<__nv_bfloat16*>(base + o) = h;
    *reinterpret_cast<__nv_bfloat16*>(base + bchunk + o) = l;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

void geometry(const Shape& s, int mode, int64_t* L, int64_t* G) {
  *L = 1;
  *G = 1;
  for (int m = 0; m < mode; ++m) *L *= s.dims[m];
  for (int m = mode + 1; m < s.N; ++m) *G *= s.dims[m];
}

int num_sms() {
  static int v = 0;
  if (v == 0) {
    int dev = 0, x = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&x, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || x <= 0) x = 148;
    cudaGetLastError();
    v = x;
  }
  return v;
}

int smem_optin_tc() {
  static int v = 0;
  if (v == 0) {
    int dev = 0, x = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&x, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || x <= 0)
      x = 227 * 1024;
    cudaGetLastError();
    v = x;
  }
  return v;
}

}  // namespace

size_t ttm_tc_scratch_bytes(int64_t max_In) {
  return (size_t)cdiv(std::max<int64_t>(max_In, 1), BKT) * 4 * 256 * BKT;
}

bool ttm_tc_supported(const Shape& s, int dtype, int mode, int64_t Ic) {
  if (dtype != CPMG_F32 || Ic < 1 || Ic > 256) return false;
  int64_t L, G;
  geometry(s, mode, &L, &G);
  const int64_t In = s.dims[mode];
  const int64_t M = mode == 0 ? G : L;
  // one launch holds tiles x batch CTAs; tensor-map coordinates are 32-bit
  return In >= 1 && M >= 1 && In < (1ll << 31) && M < (1ll << 31) && G < (1ll << 31) &&
         cdiv(M, BMT) * (mode == 0 ? 1 : G) < 0x7fffffffll;
}

int ttm_mode_tc(const Shape& s, const float* Z, int mode, const double* Rh, int64_t Ic, float* Y, void* scratch,
                int* err, cudaEvent_t ev0, cudaEvent_t ev1, bool ev_external, cudaStream_t st) {
  if (!ttm_tc_supported(s, CPMG_F32, mode, Ic) || !scratch) return CPMG_UNSUPPORTED;
  int64_t L, G;
  geometry(s, mode, &L, &G);
  const int64_t In = s.dims[mode];
  const int Npad = (int)cdiv(Ic, 16) * 16;
  const int nk = (int)cdiv(In, BKT);
  const uint32_t bchunk = (uint32_t)Npad * BKT * 2;
  unsigned char* bsplit = reinterpret_cast<unsigned char*>(scratch);
  {
    const int64_t tot = (int64_t)nk * Npad * BKT;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(tot, 256), 1024));
    k_split_rhat<<<nb, 256, 0, st>>>(Rh, Ic, In, Npad, nk, bchunk, bsplit);
    CPMG_CUDA_TRY(cudaGetLastError());
  }
  TcArgs a{};
  a.Ic = Ic;
  a.Npad = Npad;
  a.K = In;
  a.Z = Z;
  a.bsplit = bsplit;
  a.bchunk = bchunk;
  a.Y = Y;
  a.err = err;
  a.first = mode == 0;
  a.M = mode == 0 ? G : L;
  a.batch = mode == 0 ? 1 : G;
  if (mode == 0) {
    a.ldy_m = Ic;
    a.ldy_c = 1;
    a.ldy_b = 0;
  } else {
    a.ldy_m = 1;
    a.ldy_c = L;
    a.ldy_b = L * Ic;
  }
  // a tensor map when the base and the row strides are 16-byte aligned, else direct loads
  CUtensorMap tmap;
  std::memset(&tmap, 0, sizeof(tmap));
  const bool aligned = (reinterpret_cast<uintptr_t>(Z) % 16) == 0 && encode_fn() != nullptr &&
                       (mode == 0 ? (In % 4) == 0 : (L % 4) == 0);
  a.direct = 1;
  if (aligned) {
    CUresult r;
    if (mode == 0) {
      cuuint64_t dims[2] = {(cuuint64_t)In, (cuuint64_t)G};
      cuuint64_t strides[1] = {(cuuint64_t)In * 4};
      cuuint32_t box[2] = {BKT, BMT};
      cuuint32_t estr[2] = {1, 1};
      r = encode_fn()(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(Z), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
      cuuint64_t dims[3] = {(cuuint64_t)L, (cuuint64_t)In, (cuuint64_t)G};
      cuuint64_t strides[2] = {(cuuint64_t)L * 4, (cuuint64_t)L * In * 4};
      cuuint32_t box[3] = {32, BKT, 1};
      cuuint32_t estr[3] = {1, 1, 1};
      r = encode_fn()(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(Z), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    a.direct = r == CUDA_SUCCESS ? 0 : 1;
  }
  // R-hat chunks: a 2-D tensor map over the split buffer seen as rows of 64 BF16 (128 bytes),
  // Npad rows per chunk (bulk copies if it cannot be encoded)
  CUtensorMap bmap;
  std::memset(&bmap, 0, sizeof(bmap));
  a.btm = 0;
  if (encode_fn() != nullptr) {
    cuuint64_t dims[2] = {64, (cuuint64_t)nk * Npad};
    cuuint64_t strides[1] = {128};
    cuuint32_t box[2] = {64, (cuuint32_t)Npad};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode_fn()(&bmap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, bsplit, dims, strides, box, estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    a.btm = r == CUDA_SUCCESS ? 1 : 0;
  }
  // mode-1 output through TMA stores: a 2-D map over Y (Ic floats per row), 32 x 32 boxes
  CUtensorMap ymap;
  std::memset(&ymap, 0, sizeof(ymap));
  a.ytm = 0;
  if (mode == 0 && (Ic % 4) == 0 && Ic >= 32 && (reinterpret_cast<uintptr_t>(Y) % 16) == 0 && encode_fn() != nullptr) {
    cuuint64_t dims[2] = {(cuuint64_t)Ic, (cuuint64_t)G};
    cuuint64_t strides[1] = {(cuuint64_t)Ic * 4};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode_fn()(&ymap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, Y, dims, strides, box, estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                   CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    a.ytm = r == CUDA_SUCCESS ? 1 : 0;
  }
  a.mtiles = cdiv(a.M, BMT);
  a.ntiles = a.mtiles * a.batch;
  a.vec4 = mode == 0 && (Ic % 4) == 0 && (reinterpret_cast<uintptr_t>(Y) % 16) == 0;
  const int64_t grid = std::min<int64_t>(a.ntiles, num_sms());
  // tensor memory: accumulators at columns 0 and 256 when that leaves room for three K16 A
  // stages after each (Npad <= 208), else one accumulator at 0; A stages follow each
  // accumulator, an even number of them (pairs per K step), up to eight.  The parity waits need
  // at least kGroups A stages: a splitter group then never tests a barrier more than one phase
  // ahead (its own wait kGroups half-steps earlier covered the phase before).
  a.nacc = (kAccStride - Npad) / kAStageCols >= 3 ? 2 : 1;
  a.n0 = (a.nacc == 2 ? kAccStride - Npad : kTmemCols - Npad) / kAStageCols;
  a.sa = std::min(kMaxAStages, a.nacc == 2 ? 2 * a.n0 : a.n0) & ~1;
  // shared memory: one R-hat slot per A stage pair (a K step frees both with one commit), then
  // an even fp32 ring of 2..8 slots (each splitter group then consumed the previous use of a
  // slot itself)
  const size_t bslot = 2 * (size_t)bchunk;
  const size_t cap = (size_t)smem_optin_tc();
  a.sb = a.sa / 2;
  // TMA-store staging (4 warps x 2 x 4 KB, 1 KB aligned) after the R-hat ring
  const size_t ybytes = a.ytm ? 4 * 2 * 4096 + 1024 : 0;
  if (kStageBase + a.sb * bslot + ybytes > cap) return CPMG_UNSUPPORTED;
  a.sf = a.direct ? 0
                  : (int)std::min<size_t>(kMaxRing, (cap - kStageBase - a.sb * bslot - ybytes) / kF32Bytes) & ~1;
  if (a.sa < kGroups || a.sb < 2 || (!a.direct && a.sf < 2)) return CPMG_UNSUPPORTED;
  // more than half of an SM's shared memory: one CTA per SM, so the 512-column tensor-memory
  // allocation never waits for another CTA
  const size_t smem =
      std::min(cap, std::max<size_t>(kStageBase + a.sb * bslot + (size_t)a.sf * kF32Bytes + ybytes, 120 * 1024));
  cudaFuncSetAttribute(k_ttm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
  const unsigned evflags = ev_external ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (ev0) CPMG_CUDA_TRY(cudaEventRecordWithFlags(ev0, st, evflags));
  k_ttm_tc<<<(unsigned)grid, THREADS, smem, st>>>(tmap, bmap, ymap, a);
  CPMG_CUDA_TRY(cudaGetLastError());
  if (ev1) CPMG_CUDA_TRY(cudaEventRecordWithFlags(ev1, st, evflags));
  return CPMG_OK;
}

}  // namespace cpmg
