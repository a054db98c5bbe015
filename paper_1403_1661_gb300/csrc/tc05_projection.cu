// Measurement probe: the projection half of the tensor-core volume term on one
// 128-element tile, written for the two tensor-core paths of sm_103a.
//
// The volume term of Section 7.1, N(Q) = Pr cF1 + Ps cF2 + P cS, is per field a
// product R[elements x Np] += Flux[elements x cubature points] * Op^T. In the stage
// kernel the flux is produced in registers, one value per (element, point), and
// the projection consumes it at once. This probe isolates that step for N = 4
// (Np = 15 padded to 16, 36 cubature points padded to 40) with a flux that costs
// one multiply-add per value, a[e][q] = x[e] c[q] + y[e], so that what is timed is
// the hand-over of the flux to the tensor core and the product itself:
//
//   impl 0  warp-level mma.sync m16n8k8 TF32: each warp computes its 32 elements'
//           flux directly in the A-fragment layout and accumulates in registers
//           (the stage kernel's scheme, single product);
//   impl 1  tcgen05.mma kind::tf32, M = 128, N = 16, K = 8: each thread computes
//           its element's row, stores it to shared memory in the canonical K-major
//           layout (8-row by 16-byte core matrices), one thread issues the five
//           MMAs of the tile into a TMEM accumulator and commits them to an
//           mbarrier; the A tile is double-buffered, so the next tile's flux is
//           computed while the tensor core reads the previous one. After the last
//           tile each warp reads its 32 TMEM lanes back with tcgen05.ld;
//   impl 2  impl 1 through four A buffers synchronised by mbarriers only;
//   impl 3, 4  impl 1 with N = 64 or 128 (the operator's columns repeated);
//   impl 5  the flux stored to TMEM (tcgen05.st) and read by the MMA as A.
//
// All accumulate D = sum over the CTA's tiles of A_t B and write it once, so the
// timed work is flux generation plus projection; all round the operands to TF32
// the same way (cvt.rna), so their results agree up to summation order.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/swe.h"

namespace swe {
void set_last_error(const std::string& msg);  // defined with the other entry points
}

namespace {

constexpr int kRows = 128;        // elements per tile: the tcgen05 M
constexpr int kK = 40;            // cubature points per tile (36 for N = 4, padded)
constexpr int kN = 16;            // nodes (15 for N = 4, padded): the MMA N
constexpr int kKG = kK / 4;       // 16-byte chunks of a K-major row (four TF32 words)
constexpr int kThreads = 128;
constexpr int kTmemCols = 32;     // smallest TMEM allocation; D uses kN of them
constexpr int kSmemA = kRows * kK;          // words per A buffer
constexpr int kSmemB = kN * kK;             // words of B
constexpr int kSmemBytes = (2 * kSmemA + kSmemB) * 4;

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32_k8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                            uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// impl 0 -------------------------------------------------------------------
// m16n8k8 TF32 fragments (lane = 4 g + t): A a0 (g, t), a1 (g + 8, t), a2 (g, t + 4),
// a3 (g + 8, t + 4); B b0 (k = t, n = g), b1 (t + 4, g); C c0, c1 (g, 2t and 2t + 1),
// c2, c3 (g + 8, same columns).
__global__ void __launch_bounds__(kThreads) k_proj_mma(const float* __restrict__ x, const float* __restrict__ y,
                                                       const float* __restrict__ c, const float* __restrict__ b,
                                                       float* __restrict__ d, int tiles) {
  __shared__ float sc[kK];
  __shared__ uint32_t sb[kK * kN];
  for (int i = threadIdx.x; i < kK * kN; i += kThreads) sb[i] = to_tf32(__ldg(b + i));
  for (int i = threadIdx.x; i < kK; i += kThreads) sc[i] = __ldg(c + i);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  // the operator's fragments are the same for every tile: registers
  uint32_t bf[kK / 8][2][2];
  float cq[kK / 8][2];
#pragma unroll
  for (int ks = 0; ks < kK / 8; ++ks) {
    cq[ks][0] = sc[8 * ks + t];
    cq[ks][1] = sc[8 * ks + t + 4];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      bf[ks][nt][0] = sb[(8 * ks + t) * kN + 8 * nt + g];
      bf[ks][nt][1] = sb[(8 * ks + t + 4) * kN + 8 * nt + g];
    }
  }
  float acc[2][2][4] = {};
  for (int tile = 0; tile < tiles; ++tile) {
    const size_t base = ((size_t)blockIdx.x * tiles + tile) * kRows + warp * 32;
    float xr[2][2], yr[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        xr[mt][h] = __ldg(x + base + 16 * mt + 8 * h + g);
        yr[mt][h] = __ldg(y + base + 16 * mt + 8 * h + g);
      }
#pragma unroll
    for (int ks = 0; ks < kK / 8; ++ks)
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const uint32_t a0 = to_tf32(fmaf(xr[mt][0], cq[ks][0], yr[mt][0]));
        const uint32_t a1 = to_tf32(fmaf(xr[mt][1], cq[ks][0], yr[mt][1]));
        const uint32_t a2 = to_tf32(fmaf(xr[mt][0], cq[ks][1], yr[mt][0]));
        const uint32_t a3 = to_tf32(fmaf(xr[mt][1], cq[ks][1], yr[mt][1]));
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) mma_tf32_k8(acc[mt][nt], a0, a1, a2, a3, bf[ks][nt][0], bf[ks][nt][1]);
      }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const size_t r0 = (size_t)blockIdx.x * kRows + warp * 32 + 16 * mt + g;
      const int col = 8 * nt + 2 * t;
      d[r0 * kN + col] = acc[mt][nt][0];
      d[r0 * kN + col + 1] = acc[mt][nt][1];
      d[(r0 + 8) * kN + col] = acc[mt][nt][2];
      d[(r0 + 8) * kN + col + 1] = acc[mt][nt][3];
    }
}

}  // namespace

// impl 1 -------------------------------------------------------------------
namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Wait, at most limit_ns, until the phase of the given parity has completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  const unsigned long long t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// Shared-memory matrix descriptor, canonical K-major layout without swizzle: core
// matrices of 8 rows x 16 bytes stored as 128 contiguous bytes; lbo = byte distance
// between the two core matrices of one MMA's K extent, sbo = byte distance between
// adjacent 8-row groups. Fields (addresses and offsets in 16-byte units): start
// [0, 14), leading offset [16, 30), stride offset [32, 46), descriptor version 1 at
// [46, 48), base offset 0, layout type 0 (no swizzle) at [61, 64).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::tf32: D F32 (bits 4-5 = 1), A and B TF32 (bits 7-9
// and 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}
constexpr uint32_t kIdesc = idesc_tf32(kN);

__device__ __forceinline__ void mma_tc05(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate,
                                         uint32_t idesc = kIdesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy stores to shared memory, made visible to the tensor core's reads
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive 32-bit TMEM columns of the warp's 32 lanes: lane l gets row (lane
// base + l), columns [col, col + 16).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}

// NB: the MMA's N. The projection needs 16 columns; NB = 64 or 128 repeats B's
// columns (n mod 16) to time wider instructions on the same A tiles, and only the
// first 16 columns are read back.
template <int NB>
__global__ void __launch_bounds__(kThreads) k_proj_tc05(const float* __restrict__ x, const float* __restrict__ y,
                                                        const float* __restrict__ c, const float* __restrict__ b,
                                                        float* __restrict__ d, int tiles, int* status,
                                                        unsigned long long limit_ns) {
  constexpr int kCols = NB < 32 ? 32 : NB;   // TMEM columns: a power of two, at least 32
  extern __shared__ __align__(128) uint32_t smem_w[];
  uint32_t* sA = smem_w;                // [2][kSmemA] words, canonical K-major
  uint32_t* sB = smem_w + 2 * kSmemA;   // [NB * kK] words, canonical K-major
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ float sc[kK];
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  // B^T (row n = node, K = cubature point), core matrix (n / 8, q / 4) at
  // ((n / 8) kKG + q / 4) 32 words, row n % 8 at 4 words each
  for (int i = tid; i < NB * kK; i += kThreads) {
    const int n = i / kK, q = i % kK;
    sB[((n >> 3) * kKG + (q >> 2)) * 32 + (n & 7) * 4 + (q & 3)] = to_tf32(__ldg(b + q * kN + n % kN));
  }
  for (int i = tid; i < kK; i += kThreads) sc[i] = __ldg(c + i);
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    // the initialised barriers, visible to the tensor core's arrivals
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_slot;
  const uint32_t aBase = smem_addr(sA), bBase = smem_addr(sB);
  uint32_t parity[2] = {0u, 0u};   // thread 0: next phase to wait for, per buffer
  int issued = 0;                  // tiles whose MMAs were issued
  for (int tile = 0; tile < tiles; ++tile) {
    const int buf = tile & 1;
    // the MMAs that read this buffer two tiles ago must be done before it is rewritten
    if (tid == 0 && tile >= 2) {
      if (!mbar_wait(&bar[buf], parity[buf], limit_ns)) s_fail = 1;
      parity[buf] ^= 1u;
    }
    __syncthreads();
    if (s_fail) break;
    {
      const int r = tid;
      const size_t row = ((size_t)blockIdx.x * tiles + tile) * kRows + r;
      const float xr = __ldg(x + row), yr = __ldg(y + row);
      uint32_t* a = sA + buf * kSmemA + (r >> 3) * kKG * 32 + (r & 7) * 4;
#pragma unroll
      for (int kg = 0; kg < kKG; ++kg) {
        uint4 v;
        v.x = to_tf32(fmaf(xr, sc[4 * kg + 0], yr));
        v.y = to_tf32(fmaf(xr, sc[4 * kg + 1], yr));
        v.z = to_tf32(fmaf(xr, sc[4 * kg + 2], yr));
        v.w = to_tf32(fmaf(xr, sc[4 * kg + 3], yr));
        *reinterpret_cast<uint4*>(a + kg * 32) = v;
      }
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
#pragma unroll
      for (int ks = 0; ks < kK / 8; ++ks) {
        // one MMA covers K = 8 = two core matrices along K (256 bytes further per step)
        const uint64_t ad = smem_desc(aBase + (buf * kSmemA + ks * 2 * 32) * 4, 128, kKG * 128);
        const uint64_t bd = smem_desc(bBase + (ks * 2 * 32) * 4, 128, kKG * 128);
        mma_tc05(tmem, ad, bd, (tile > 0 || ks > 0) ? 1u : 0u, idesc_tf32(NB));
      }
      mma_commit(&bar[buf]);
    }
    issued = tile + 1;
  }
  // the outstanding commits: the last two tiles (one if only one was issued)
  if (tid == 0) {
    for (int tile = issued >= 2 ? issued - 2 : 0; tile < issued; ++tile) {
      const int buf = tile & 1;
      if (!mbar_wait(&bar[buf], parity[buf], limit_ns)) s_fail = 1;
      parity[buf] ^= 1u;
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (!s_fail) {
    uint32_t v[16];
    tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16), v);
    float* out = d + ((size_t)blockIdx.x * kRows + tid) * kN;
#pragma unroll
    for (int j = 0; j < 16; ++j) out[j] = __uint_as_float(v[j]);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
  if (tid == 0) status[blockIdx.x] = s_fail ? SWE_ETIMEOUT : SWE_OK;
}

// impl 2: the same product, pipelined through kBufs A buffers with mbarriers only
// (no CTA barrier in the loop). Every thread writes its row of buffer (t mod kBufs)
// and arrives on full[buf] (count 128); thread 0 waits for the full buffer, issues
// the five MMAs and commits them to empty[buf]; a thread waits on empty[buf] only
// before it rewrites the buffer kBufs tiles later. Warps thus run up to kBufs tiles
// ahead of the tensor core.
constexpr int kBufs = 4;
constexpr int kSmemBytes2 = (kBufs * kSmemA + kSmemB) * 4;

// arrive on a barrier; returns the barrier state token (unused by the callers)
__device__ __forceinline__ unsigned long long mbar_arrive(uint64_t* bar) {
  unsigned long long state;
  asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(smem_addr(bar)) : "memory");
  return state;
}

__global__ void __launch_bounds__(kThreads) k_proj_tc05_pipe(const float* __restrict__ x,
                                                             const float* __restrict__ y,
                                                             const float* __restrict__ c,
                                                             const float* __restrict__ b, float* __restrict__ d,
                                                             int tiles, int* status, unsigned long long limit_ns) {
  extern __shared__ __align__(128) uint32_t smem_w[];
  uint32_t* sA = smem_w;                     // [kBufs][kSmemA] words, canonical K-major
  uint32_t* sB = smem_w + kBufs * kSmemA;    // [kSmemB] words, canonical K-major
  __shared__ __align__(8) uint64_t full[kBufs];
  __shared__ __align__(8) uint64_t empty[kBufs];
  __shared__ uint32_t tmem_slot;
  __shared__ float sc[kK];
  __shared__ volatile int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < kN * kK; i += kThreads) {
    const int n = i / kK, q = i % kK;
    sB[((n >> 3) * kKG + (q >> 2)) * 32 + (n & 7) * 4 + (q & 3)] = to_tf32(__ldg(b + q * kN + n));
  }
  for (int i = tid; i < kK; i += kThreads) sc[i] = __ldg(c + i);
  if (tid == 0) {
    for (int i = 0; i < kBufs; ++i) {
      mbar_init(&full[i], kThreads);
      mbar_init(&empty[i], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_slot;
  const uint32_t aBase = smem_addr(sA), bBase = smem_addr(sB);
  int issued = 0;   // thread 0: tiles whose MMAs were committed
  for (int tile = 0; tile < tiles; ++tile) {
    const int buf = tile % kBufs;
    const uint32_t use = (uint32_t)(tile / kBufs);
    if (use > 0 && !mbar_wait(&empty[buf], (use - 1) & 1u, limit_ns)) s_fail = 1;
    if (s_fail) break;
    {
      const int r = tid;
      const size_t row = ((size_t)blockIdx.x * tiles + tile) * kRows + r;
      const float xr = __ldg(x + row), yr = __ldg(y + row);
      uint32_t* a = sA + buf * kSmemA + (r >> 3) * kKG * 32 + (r & 7) * 4;
#pragma unroll
      for (int kg = 0; kg < kKG; ++kg) {
        uint4 v;
        v.x = to_tf32(fmaf(xr, sc[4 * kg + 0], yr));
        v.y = to_tf32(fmaf(xr, sc[4 * kg + 1], yr));
        v.z = to_tf32(fmaf(xr, sc[4 * kg + 2], yr));
        v.w = to_tf32(fmaf(xr, sc[4 * kg + 3], yr));
        *reinterpret_cast<uint4*>(a + kg * 32) = v;
      }
    }
    fence_async_smem();
    (void)mbar_arrive(&full[buf]);
    if (tid == 0) {
      if (!mbar_wait(&full[buf], use & 1u, limit_ns)) {
        s_fail = 1;
        break;
      }
      fence_after_sync();
#pragma unroll
      for (int ks = 0; ks < kK / 8; ++ks) {
        const uint64_t ad = smem_desc(aBase + (buf * kSmemA + ks * 2 * 32) * 4, 128, kKG * 128);
        const uint64_t bd = smem_desc(bBase + (ks * 2 * 32) * 4, 128, kKG * 128);
        mma_tc05(tmem, ad, bd, (tile > 0 || ks > 0) ? 1u : 0u);
      }
      mma_commit(&empty[buf]);
      issued = tile + 1;
    }
  }
  // thread 0: the commits nobody waited for (the last kBufs tiles)
  if (tid == 0) {
    for (int tile = issued > kBufs ? issued - kBufs : 0; tile < issued; ++tile)
      if (!mbar_wait(&empty[tile % kBufs], (uint32_t)(tile / kBufs) & 1u, limit_ns)) s_fail = 1;
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (!s_fail) {
    uint32_t v[16];
    tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16), v);
    float* out = d + ((size_t)blockIdx.x * kRows + tid) * kN;
#pragma unroll
    for (int j = 0; j < 16; ++j) out[j] = __uint_as_float(v[j]);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  if (tid == 0) status[blockIdx.x] = s_fail ? SWE_ETIMEOUT : SWE_OK;
}

// impl 5: the flux goes from registers straight into TMEM (tcgen05.st, one lane per
// element, 32-bit columns = cubature points) and the MMA reads A from TMEM: no
// shared-memory tile and no proxy fence. TMEM columns: D [0, 16), A buffer b at
// [32 + 40 b, 72 + 40 b).
constexpr int kTmemColsA = 128;

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}

__device__ __forceinline__ void mma_tc05_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}"
      ::"r"(tmem_d), "r"(tmem_a), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__global__ void __launch_bounds__(kThreads) k_proj_tc05_tmem(const float* __restrict__ x,
                                                             const float* __restrict__ y,
                                                             const float* __restrict__ c,
                                                             const float* __restrict__ b, float* __restrict__ d,
                                                             int tiles, int* status, unsigned long long limit_ns) {
  __shared__ __align__(128) uint32_t sB[kSmemB];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ float sc[kK];
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < kN * kK; i += kThreads) {
    const int n = i / kK, q = i % kK;
    sB[((n >> 3) * kKG + (q >> 2)) * 32 + (n & 7) * 4 + (q & 3)] = to_tf32(__ldg(b + q * kN + n));
  }
  for (int i = tid; i < kK; i += kThreads) sc[i] = __ldg(c + i);
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kTmemColsA)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_slot;
  const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
  const uint32_t bBase = smem_addr(sB);
  uint32_t parity[2] = {0u, 0u};
  int issued = 0;
  for (int tile = 0; tile < tiles; ++tile) {
    const int buf = tile & 1;
    if (tid == 0 && tile >= 2) {
      if (!mbar_wait(&bar[buf], parity[buf], limit_ns)) s_fail = 1;
      parity[buf] ^= 1u;
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (s_fail) break;
    {
      const size_t row = ((size_t)blockIdx.x * tiles + tile) * kRows + tid;
      const float xr = __ldg(x + row), yr = __ldg(y + row);
#pragma unroll
      for (int ks = 0; ks < kK / 8; ++ks) {
        uint32_t v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = to_tf32(fmaf(xr, sc[8 * ks + j], yr));
        tmem_st8(tmem + lane_base + 32 + 40 * buf + 8 * ks, v);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
#pragma unroll
      for (int ks = 0; ks < kK / 8; ++ks) {
        const uint64_t bd = smem_desc(bBase + (ks * 2 * 32) * 4, 128, kKG * 128);
        mma_tc05_ta(tmem, tmem + 32 + 40 * buf + 8 * ks, bd, (tile > 0 || ks > 0) ? 1u : 0u);
      }
      mma_commit(&bar[buf]);
    }
    issued = tile + 1;
  }
  if (tid == 0) {
    for (int tile = issued >= 2 ? issued - 2 : 0; tile < issued; ++tile) {
      const int buf = tile & 1;
      if (!mbar_wait(&bar[buf], parity[buf], limit_ns)) s_fail = 1;
      parity[buf] ^= 1u;
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (!s_fail) {
    uint32_t v[16];
    tmem_ld16(tmem + lane_base, v);
    float* out = d + ((size_t)blockIdx.x * kRows + tid) * kN;
#pragma unroll
    for (int j = 0; j < 16; ++j) out[j] = __uint_as_float(v[j]);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemColsA) : "memory");
  if (tid == 0) status[blockIdx.x] = s_fail ? SWE_ETIMEOUT : SWE_OK;
}

int fail_probe(int code, const std::string& msg) {
  swe::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" int swe_tc_projection_probe(int32_t impl, int32_t nctas, int32_t tiles_per_cta, const float* dev_x,
                                       const float* dev_y, const float* dev_c, const float* dev_b, float* dev_d,
                                       int32_t* dev_status, void* stream) {
  if (impl < 0 || impl > 5) return fail_probe(SWE_EINVAL, "swe_tc_projection_probe: impl must be 0 to 5");
  if (nctas < 1 || tiles_per_cta < 1 || (int64_t)nctas * tiles_per_cta * kRows > INT32_MAX)
    return fail_probe(SWE_EINVAL, "swe_tc_projection_probe: need nctas, tiles_per_cta >= 1 and rows < 2^31");
  if (!dev_x || !dev_y || !dev_c || !dev_b || !dev_d || (impl > 0 && !dev_status))
    return fail_probe(SWE_EINVAL, "swe_tc_projection_probe: NULL device pointer");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (impl == 0) {
    k_proj_mma<<<nctas, kThreads, 0, st>>>(dev_x, dev_y, dev_c, dev_b, dev_d, tiles_per_cta);
  } else if (impl == 1) {
    k_proj_tc05<kN><<<nctas, kThreads, kSmemBytes, st>>>(dev_x, dev_y, dev_c, dev_b, dev_d, tiles_per_cta,
                                                         reinterpret_cast<int*>(dev_status), 1000000000ull);
  } else if (impl == 5) {
    k_proj_tc05_tmem<<<nctas, kThreads, 0, st>>>(dev_x, dev_y, dev_c, dev_b, dev_d, tiles_per_cta,
                                                 reinterpret_cast<int*>(dev_status), 1000000000ull);
  } else if (impl == 3 || impl == 4) {
    const int nb = impl == 3 ? 64 : 128;
    const int bytes = (2 * kSmemA + nb * kK) * 4;
    cudaError_t ea = impl == 3
                         ? cudaFuncSetAttribute(k_proj_tc05<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
                         : cudaFuncSetAttribute(k_proj_tc05<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (ea != cudaSuccess)
      return fail_probe(SWE_ECUDA, std::string("swe_tc_projection_probe: shared memory: ") + cudaGetErrorString(ea));
    if (impl == 3)
      k_proj_tc05<64><<<nctas, kThreads, bytes, st>>>(dev_x, dev_y, dev_c, dev_b, dev_d, tiles_per_cta,
                                                      reinterpret_cast<int*>(dev_status), 1000000000ull);
    else
      k_proj_tc05<128><<<nctas, kThreads, bytes, st>>>(dev_x, dev_y, dev_c, dev_b, dev_d, tiles_per_cta,
                                                       reinterpret_cast<int*>(dev_status), 1000000000ull);
  } else {
    const cudaError_t ea =
        cudaFuncSetAttribute(k_proj_tc05_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes2);
    if (ea != cudaSuccess)
      return fail_probe(SWE_ECUDA, std::string("swe_tc_projection_probe: shared memory: ") + cudaGetErrorString(ea));
    k_proj_tc05_pipe<<<nctas, kThreads, kSmemBytes2, st>>>(dev_x, dev_y, dev_c, dev_b, dev_d, tiles_per_cta,
                                                           reinterpret_cast<int*>(dev_status), 1000000000ull);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail_probe(SWE_ECUDA, std::string("swe_tc_projection_probe: launch: ") + cudaGetErrorString(e));
  return SWE_OK;
}
