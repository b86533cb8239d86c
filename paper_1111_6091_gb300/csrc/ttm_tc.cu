// n-mode products Y = Z x_n R-hat on tcgen05 tensor cores (Eq. ctensor_transformed).
//
// Each mode product is a GEMM whose tensor-core M dimension is a large index of Z and whose
// N dimension is the coarse size Ic (<= 256), with L = prod_{m<n} I_m, G = prod_{m>n} I_m:
//   n = 1 : Y(c, g)    = sum_k R-hat(c, k) Z(k, g)     D(g, c), A = Z tile (K-major)
//   n > 1 : Y(l, c, g) = sum_k Z(l, k, g) R-hat(c, k)  D(l, c), A = Z tile (MN-major), per g
// B is R-hat with c contiguous (MN-major) in both cases.
//
// Precision (split BF16): every float x is hi + lo with hi = bf16(x), lo = bf16(x - hi).  The
// products hi*hi + hi*lo + lo*hi are accumulated in FP32 in tensor memory; the dropped lo*lo
// term and the rounding of lo leave a relative error near 2^-16 per product.
//
// Persistent CTAs of 480 threads, one per SM, walk 128-row output tiles:
//   warp 0      producer: fp32 tiles of Z by cp.async.bulk.tensor (128-byte swizzle)
//   warps 1..8  split the fp32 tile into BF16 hi / lo in the canonical no-swizzle core-matrix
//               layout (or load it straight from global memory when the tensor's strides do
//               not suit a tensor map)
//   warp 9      allocates tensor memory (two accumulators of 256 columns); one lane issues
//               tcgen05.mma into the accumulator of the current tile
//   warps 10-13 drain the other accumulator into Y while the next tile is computed
//   warp 14     producer: pre-split R-hat chunks by cp.async.bulk
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

constexpr int BMT = 128;      // tensor-core M tile (TMEM lanes)
constexpr int BKT = 32;       // K per pipeline stage (two MMA K steps)
constexpr int kConvWarps = 8;                   // warps splitting fp32 -> BF16 (warps 1..8)
constexpr int kMmaWarp = 1 + kConvWarps;        // tensor-memory owner and MMA issuer
constexpr int kEpiWarp0 = kMmaWarp + 1;         // four epilogue warps
constexpr int kBWarp = kEpiWarp0 + 4;           // R-hat chunk producer
constexpr int THREADS = 32 * (kBWarp + 1);
constexpr int kUnitsPerThread = 512 / (32 * kConvWarps);  // 16-byte core-matrix rows per stage
constexpr int kTmemCols = 256;
constexpr uint32_t kF32Bytes = BMT * BKT * 4;   // fp32 staging of one stage
constexpr uint32_t kAHalf = BMT * BKT * 2;      // one BF16 term of A
constexpr int kStageBase = 1024;                // 128-byte swizzle wants 1 KB alignment

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

// bounded wait: false after ~2 s without the phase completing
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  if (bar_try(bar, parity)) return true;
  const uint64_t t0 = gtime();
  while (true) {
    if (bar_try(bar, parity)) return true;
    if (gtime() - t0 > 2000000000ull) return false;
  }
}

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

// shared-memory matrix descriptor: start, leading / stride byte offsets, tcgen05 version,
// no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
               "l"(da), "l"(db), "r"(idesc), "r"(acc)
               : "memory");
}

// x -> (hi, lo) for 8 floats, packed as bf16 pairs
__device__ __forceinline__ void split8(const float* x, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * i]), h1 = __float2bfloat16_rn(x[2 * i + 1]);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * i] - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * i + 1] - __bfloat162float(h1));
    h[i] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
    l[i] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// byte offset of 16-byte chunk `chunk` of 128-byte row `row` under the 128-byte swizzle
__device__ __forceinline__ uint32_t sw128(int row, int chunk) {
  return (uint32_t)row * 128u + (uint32_t)((chunk ^ (row & 7)) << 4);
}

struct TcArgs {
  int first;            // 1: mode 1 (A K-major), 0: later mode (A MN-major)
  int direct;           // 1: converters load Z from global memory (no tensor map)
  int sf, sm;           // slots of the fp32 ring and of the MMA-operand ring
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

__device__ __forceinline__ bool failed(const int* fail) { return *reinterpret_cast<const volatile int*>(fail) != 0; }

// Persistent: CTA b handles tiles b, b + gridDim.x, ...  Two rings of shared memory: fp32 tiles
// of Z (freed as soon as they are split, so Z loads run several stages ahead) and MMA operands
// (BF16 hi / lo of the Z tile and the R-hat chunk, freed by the MMA commit).  Two tensor-memory
// accumulators let the epilogue of one tile overlap the main loop of the next.
__global__ void __launch_bounds__(THREADS, 1) k_ttm_tc(const __grid_constant__ CUtensorMap tmap, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int SF = a.sf, SM = a.sm;
  uint64_t* ffull = reinterpret_cast<uint64_t*>(smem);  // fp32 tile landed
  uint64_t* fempty = ffull + 8;                          // fp32 tile read by the splitters
  uint64_t* mfull = fempty + 8;                          // R-hat chunk landed (slot claimed)
  uint64_t* conv = mfull + 8;                            // BF16 split written
  uint64_t* mempty = conv + 8;                           // MMAs reading the slot completed
  uint64_t* tfull = mempty + 8;                          // [2] accumulator complete
  uint64_t* tempty = tfull + 2;                          // [2] accumulator drained
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 512);
  int* fail = reinterpret_cast<int*>(smem + 520);
  const uint32_t mslot = 2 * kAHalf + 2 * a.bchunk;
  unsigned char* fring = smem + kStageBase;
  unsigned char* mring = fring + (size_t)SF * kF32Bytes;
  const int nk = (int)((a.K + BKT - 1) / BKT);
  const uint32_t a_lbo = a.first ? 128u : (uint32_t)(BMT / 8) * 128u;
  const uint32_t a_sbo = a.first ? (uint32_t)(BKT / 8) * 128u : 128u;
  const uint32_t b_lbo = (uint32_t)(a.Npad / 8) * 128u, b_sbo = 128u;

  if (t == 0) {
    for (int s = 0; s < 8; ++s) {
      bar_init(&ffull[s], 1);
      bar_init(&fempty[s], kConvWarps);
      bar_init(&mfull[s], 1);
      bar_init(&conv[s], kConvWarps);
      bar_init(&mempty[s], 1);
    }
    for (int j = 0; j < 2; ++j) {
      bar_init(&tfull[j], 1);
      bar_init(&tempty[j], 4);
    }
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(2 * kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (warp == 0 || warp == kBWarp) {
    // ------------------------------------------------------------ producers
    // warp 0: fp32 tiles of Z (tensor map); warp 10: R-hat chunks into the operand ring
    const bool zp = warp == 0;
    if (lane == 0 && !(zp && a.direct)) {
      const int S = zp ? SF : SM;
      uint64_t* fullb = zp ? ffull : mfull;
      uint64_t* emptyb = zp ? fempty : mempty;
      int it = 0;
      for (int64_t tile = blockIdx.x; tile < a.ntiles && !failed(fail); tile += gridDim.x) {
        const int64_t b = tile / a.mtiles;
        const int m0 = (int)((tile % a.mtiles) * BMT);
        for (int kc = 0; kc < nk; ++kc, ++it) {
          const int s = it % S;
          if (it >= S && !bar_wait(&emptyb[s], (uint32_t)(((it / S) - 1) & 1))) {
            atomicOr(fail, 1);
            break;
          }
          const int k0 = kc * BKT;
          if (zp) {
            unsigned char* st = fring + (size_t)s * kF32Bytes;
            bar_arrive_tx(&fullb[s], kF32Bytes);
            if (a.first) {
              // box {BKT along k, BMT along g}: 128 rows of 128 bytes
              asm volatile(
                  "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                  "[%4];" ::"r"(su32(st)),
                  "l"(&tmap), "r"(k0), "r"(m0), "r"(su32(&fullb[s]))
                  : "memory");
            } else {
              // four boxes {32 along l, BKT along k, 1}: each 32 rows (k) of 128 bytes (l)
              for (int q = 0; q < BMT / 32; ++q)
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                    "%4}], [%5];" ::"r"(su32(st + q * 4096)),
                    "l"(&tmap), "r"(m0 + 32 * q), "r"(k0), "r"((int)b), "r"(su32(&fullb[s]))
                    : "memory");
            }
          } else {
            unsigned char* st = mring + (size_t)s * mslot;
            bar_arrive_tx(&fullb[s], 2 * a.bchunk);
            const unsigned char* src = a.bsplit + (size_t)kc * 2 * a.bchunk;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    su32(st + 2 * kAHalf)),
                "l"(src), "r"(2 * a.bchunk), "r"(su32(&fullb[s]))
                : "memory");
          }
        }
      }
      // the CTA may not exit while a copy is still in flight
      for (int j = (it > S ? it - S : 0); j < it; ++j)
        if (!bar_wait(&fullb[j % S], (uint32_t)((j / S) & 1))) atomicOr(fail, 1);
    }
  } else if (warp <= kConvWarps) {
    // ------------------------------------------------------------ split fp32 -> BF16 hi / lo
    const int ct = t - 32;  // 0 .. 32 * kConvWarps - 1
    int it = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x) {
      const int64_t b = tile / a.mtiles;
      const int64_t m0 = (tile % a.mtiles) * BMT;
      for (int kc = 0; kc < nk; ++kc, ++it) {
        const int sf = SF > 0 ? it % SF : 0, sm = it % SM;
        const int64_t k0 = (int64_t)kc * BKT;
        float x[kUnitsPerThread][8];
        if (a.direct) {
          // issue the loads before waiting for the slot
#pragma unroll
          for (int j = 0; j < kUnitsPerThread; ++j) {
            const int u = ct + 32 * kConvWarps * j;
            if (a.first) {
              const int r = ((u >> 5) << 3) + (u & 7), kq = (u >> 3) & 3;
              const int64_t m = m0 + r;
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const int64_t k = k0 + kq * 8 + i;
                x[j][i] = (m < a.M && k < a.K) ? __ldg(a.Z + k + a.K * m) : 0.f;
              }
            } else {
              const int r8 = (u >> 3) & 15;
              const int64_t k = k0 + ((u >> 7) << 3) + (u & 7);
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const int64_t m = m0 + r8 * 8 + i;
                x[j][i] = (m < a.M && k < a.K) ? __ldg(a.Z + m + a.M * k + a.M * a.K * b) : 0.f;
              }
            }
          }
        } else {
          if (failed(fail) || !bar_wait(&ffull[sf], (uint32_t)((it / SF) & 1))) {
            atomicOr(fail, 1);
            ok = false;
            break;
          }
          const unsigned char* st = fring + (size_t)sf * kF32Bytes;
#pragma unroll
          for (int j = 0; j < kUnitsPerThread; ++j) {
            const int u = ct + 32 * kConvWarps * j;
            const unsigned char *p0, *p1;
            if (a.first) {
              const int r = (u >> 5) * 8 + (u & 7), kq = (u >> 3) & 3;
              p0 = st + sw128(r, 2 * kq);
              p1 = st + sw128(r, 2 * kq + 1);
            } else {
              const int r8 = (u >> 3) & 15, k = ((u >> 7) << 3) + (u & 7);
              const unsigned char* sub = st + (r8 >> 2) * 4096;
              p0 = sub + sw128(k, (r8 & 3) * 2);
              p1 = sub + sw128(k, (r8 & 3) * 2 + 1);
            }
            const float4 v0 = *reinterpret_cast<const float4*>(p0);
            const float4 v1 = *reinterpret_cast<const float4*>(p1);
            x[j][0] = v0.x; x[j][1] = v0.y; x[j][2] = v0.z; x[j][3] = v0.w;
            x[j][4] = v1.x; x[j][5] = v1.y; x[j][6] = v1.z; x[j][7] = v1.w;
          }
        }
        // the operand slot is free once its R-hat chunk has landed (claimed by the producer)
        if (failed(fail) || !bar_wait(&mfull[sm], (uint32_t)((it / SM) & 1))) {
          atomicOr(fail, 1);
          ok = false;
          break;
        }
        unsigned char* hi = mring + (size_t)sm * mslot;
        unsigned char* lo = hi + kAHalf;
        uint4 h[kUnitsPerThread], l[kUnitsPerThread];
#pragma unroll
        for (int j = 0; j < kUnitsPerThread; ++j) split8(x[j], h[j], l[j]);
        if (!a.direct) {
          __syncwarp();
          if (lane == 0) bar_arrive(&fempty[sf]);
        }
#pragma unroll
        for (int j = 0; j < kUnitsPerThread; ++j) {
          const int u = ct + 32 * kConvWarps * j;
          uint32_t o;
          if (a.first) {
            // unit = (row r, 8 consecutive k): one 16-byte core-matrix row of the K-major tile
            o = (uint32_t)(u >> 5) * a_sbo + (uint32_t)((u >> 3) & 3) * a_lbo + (uint32_t)(u & 7) * 16u;
          } else {
            // unit = (8 consecutive l, one k): one 16-byte core-matrix row of the MN-major tile
            const int k = ((u >> 7) << 3) + (u & 7);
            o = (uint32_t)((u >> 3) & 15) * a_sbo + (uint32_t)(k >> 3) * a_lbo + (uint32_t)(k & 7) * 16u;
          }
          *reinterpret_cast<uint4*>(hi + o) = h[j];
          *reinterpret_cast<uint4*>(lo + o) = l[j];
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) bar_arrive(&conv[sm]);
      }
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      // D F32, A and B BF16, A major per mode, B MN-major, N = Npad, M = 128
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((a.first ? 0u : 1u) << 15) | (1u << 16) |
                             ((uint32_t)(a.Npad >> 3) << 17) | ((uint32_t)(BMT >> 4) << 24);
      int it = 0, i = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x, ++i) {
        const int buf = i & 1;
        if (i >= 2 && (failed(fail) || !bar_wait(&tempty[buf], (uint32_t)(((i >> 1) - 1) & 1)))) {
          atomicOr(fail, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(buf * kTmemCols);
        for (int kc = 0; kc < nk; ++kc, ++it) {
          const int s = it % SM;
          const uint32_t par = (uint32_t)((it / SM) & 1);
          if (failed(fail) || !bar_wait(&conv[s], par) || !bar_wait(&mfull[s], par)) {
            atomicOr(fail, 1);
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t ahi = su32(mring + (size_t)s * mslot), alo = ahi + kAHalf;
          const uint32_t bhi = ahi + 2 * kAHalf, blo = bhi + a.bchunk;
#pragma unroll
          for (int kk = 0; kk < BKT / 16; ++kk) {
            const uint32_t ao = kk * 2 * a_lbo, bo = kk * 2 * b_lbo;
            const uint64_t dAh = sdesc(ahi + ao, a_lbo, a_sbo), dAl = sdesc(alo + ao, a_lbo, a_sbo);
            const uint64_t dBh = sdesc(bhi + bo, b_lbo, b_sbo), dBl = sdesc(blo + bo, b_lbo, b_sbo);
            mma_bf16(d, dAh, dBh, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
            mma_bf16(d, dAh, dBl, idesc, 1u);
            mma_bf16(d, dAl, dBh, idesc, 1u);
          }
          // the slot may be refilled once these MMAs have read it
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           su32(&mempty[s]))
                       : "memory");
        }
        // accumulator `buf` is complete once every MMA issued so far has finished
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         su32(&tfull[buf]))
                     : "memory");
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue (4 warps): TMEM -> Y
    const int quarter = warp & 3;  // a warp reaches TMEM lanes 32 * (warp id mod 4) .. + 31
    int i = 0;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++i) {
      const int buf = i & 1;
      bool ok = !failed(fail) && bar_wait(&tfull[buf], (uint32_t)((i >> 1) & 1));
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) atomicOr(fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int64_t b = tile / a.mtiles;
      const int64_t row = (tile % a.mtiles) * BMT + 32 * quarter + lane;
      float* y = a.Y + b * a.ldy_b + row * a.ldy_m;
      const uint32_t base = tmem + (uint32_t)(buf * kTmemCols) + ((uint32_t)(32 * quarter) << 16);
      for (int c0 = 0; c0 < a.Npad; c0 += 16) {
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(base + (uint32_t)c0));
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
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) bar_arrive(&tempty[buf]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTmemCols) : "memory");
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
  a.mtiles = cdiv(a.M, BMT);
  a.ntiles = a.mtiles * a.batch;
  a.vec4 = mode == 0 && (Ic % 4) == 0 && (reinterpret_cast<uintptr_t>(Y) % 16) == 0;
  const int64_t grid = std::min<int64_t>(a.ntiles, num_sms());
  // operand ring: 3 slots (4 when they are small); fp32 ring: the rest of shared memory, 2..8
  const size_t mslot = 2 * kAHalf + 2 * (size_t)bchunk;
  const size_t cap = (size_t)smem_optin_tc();
  a.sm = mslot <= 32768 ? 4 : 3;
  if (kStageBase + a.sm * mslot + (a.direct ? 0 : 2 * kF32Bytes) > cap) a.sm = 2;
  a.sf = a.direct ? 0 : (int)std::min<size_t>(8, (cap - kStageBase - a.sm * mslot) / kF32Bytes);
  if (!a.direct && a.sf < 2) return CPMG_UNSUPPORTED;
  // more than half of an SM's shared memory: one CTA per SM, so the 512-column tensor-memory
  // allocation never waits for another CTA
  const size_t smem =
      std::min(cap, std::max<size_t>(kStageBase + a.sm * mslot + (size_t)a.sf * kF32Bytes, 120 * 1024));
  cudaFuncSetAttribute(k_ttm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
  const unsigned evflags = ev_external ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (ev0) CPMG_CUDA_TRY(cudaEventRecordWithFlags(ev0, st, evflags));
  k_ttm_tc<<<(unsigned)grid, THREADS, smem, st>>>(tmap, a);
  CPMG_CUDA_TRY(cudaGetLastError());
  if (ev1) CPMG_CUDA_TRY(cudaEventRecordWithFlags(ev1, st, evflags));
  return CPMG_OK;
}

}  // namespace cpmg
