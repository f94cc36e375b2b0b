// Nonlocal projector step on the 5th-generation tensor cores (tcgen05), BF16
// operands with FP32 accumulation in tensor memory (Eq. pauli_ks, the separable
// term sum_ij D_ij |beta_i><beta_j|; the products p_ij = <beta|psi> are the
// "becp" of Sec. "New parallelization levels"):
//
//   becp   = beta^H psi            (M = 2P, N = 2nb, K = npw)
//   becp'  = D becp                (diagonal D in the reduction, full D as a GEMM)
//   hpsi  += beta becp'            (M = npw, N = 2nb, K = 2P)
//
// Complex products become one real GEMM each by interleaving real and
// imaginary parts:
//   becp:  A1[2p+c][G] = (Re,Im) beta_p(G),  B1[2b+c][G] = (Re,Im) psi_b(G);
//          C1[2p..2p+1][2b..2b+1] holds the four real products, combined as
//          Re = C[2p][2b] + C[2p+1][2b+1], Im = C[2p][2b+1] - C[2p+1][2b].
//   back:  A2[G][2p+c] = (Re,Im) beta_p(G),
//          B2[2b][2p] = Re p', B2[2b][2p+1] = -Im p',
//          B2[2b+1][2p] = Im p', B2[2b+1][2p+1] = Re p',
//          so that C2[G][2b] = Re (beta p')_b(G) and C2[G][2b+1] = Im.
// Both operands are K-major.  Each operand is stored as [hi | lo] with
// hi = bf16(x), lo = bf16(x - hi); with terms = 3 the GEMM accumulates
// hi*hi + hi*lo + lo*hi (about 16 significant bits), with terms = 1 hi*hi.
//
// Kernel: 128 threads, one 128 x 256 output tile per CTA (tcgen05.mma
// cta_group::1, M = 128, N = 256, K = 16 per instruction), 4-stage TMA ring of
// 64-wide K slabs with 128-byte swizzle, one elected thread producing TMA
// loads, one issuing MMAs, then all four warps draining TMEM with tcgen05.ld.
// Every mbarrier wait is bounded (about one second of %globaltimer); on
// timeout the kernel records PWH_ERR_TIMEOUT in a device word, stops issuing,
// waits (bounded) for the copies it started, frees its tensor memory and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "gemm.cuh"

namespace pwh {

constexpr int TC_BM = 128, TC_BN = 256, TC_BK = 64, TC_STAGES = 4;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;            // 16 KB
constexpr int TC_B_BYTES = TC_BN * TC_BK * 2;            // 32 KB
constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;  // 48 KB
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr int TC_TMEM_COLS = 256;
constexpr unsigned long long TC_WAIT_NS = 1000000000ull;  // 1 s

struct TcArgs {
  int M, N;          // output rows (A rows) and columns (B rows)
  int kb_seg;        // 64-wide K blocks per [hi|lo] segment
  int terms;         // 1: hi*hi; 3: hi*hi + hi*lo + lo*hi
  int kb_per_split;  // logical K blocks per blockIdx.z
  float* part;       // mode 0: FP32 out[z][n][m]
  float2* vnl;       // mode 1: vnl[b*ldv + m] = (C[m][2b], C[m][2b+1])
  int64_t ldv;
  int nb;
  int* err;          // device error word
  // sliced operands: product t multiplies A segment oz_a[t] by B segment
  // oz_b[t]; oz = 1: blockIdx.z = (K chunk, product), each partial one product
  // (FP64-equivalent GEMM); oz = 2 (FP32-equivalent GEMM): blockIdx.z < z_rest
  // takes kb_per_split blocks of products 1.., the others kps0 blocks of
  // product 0
  int oz;
  unsigned char oz_a[64], oz_b[64];
  int z_rest, kps0;
};

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; also gives up early once *abort is raised by another role.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try(bar, parity)) return true;
    if (abort && *abort) return false;
    if (gtimer() - t0 > TC_WAIT_NS) return false;
  }
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(su32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}
// Shared-memory matrix descriptor: K-major operand tile, rows of 128 bytes,
// 128-byte swizzle, 8-row groups 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
  d |= (uint64_t)1 << 46;                  // version
  d |= (uint64_t)2 << 61;                  // SWIZZLE_128B
  return d;
}
// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// K blocks [kb0, kb_end) of grid slice z: sliced operands (oz = 1: z = chunk x
// products + product; oz = 2: the long ranges of products 1.. first, then the
// short ranges of product 0) or plain split-K ranges.
__device__ __forceinline__ void tc_krange(const TcArgs& args, int z, int& kb0, int& kb_end) {
  const int kb_total = args.terms * args.kb_seg;
  if (args.oz == 1) {
    kb0 = (z % args.terms) * args.kb_seg + (z / args.terms) * args.kb_per_split;
    kb_end = min(kb_total, kb0 + args.kb_per_split);
  } else if (args.oz == 2 && z < args.z_rest) {
    kb0 = args.kb_seg + z * args.kb_per_split;
    kb_end = min(kb_total, kb0 + args.kb_per_split);
  } else if (args.oz == 2) {
    kb0 = (z - args.z_rest) * args.kps0;
    kb_end = min(args.kb_seg, kb0 + args.kps0);
  } else {
    kb0 = z * args.kb_per_split;
    kb_end = min(kb_total, kb0 + args.kb_per_split);
  }
}

// Logical K block kb -> (A column, B column) in elements, for the [hi|lo]
// operand layout: term 0 = (hi, hi), term 1 = (hi, lo), term 2 = (lo, hi).
__device__ __forceinline__ void kb_coords(int kb, int kb_seg, int& xa, int& xb) {
  int t = kb / kb_seg, r = kb - t * kb_seg;
  int sa = (t == 2) ? 1 : 0, sb = (t == 1) ? 1 : 0;
  xa = (sa * kb_seg + r) * TC_BK;
  xb = (sb * kb_seg + r) * TC_BK;
}

// Persistent, warp-specialised form: one CTA per SM walks the output tiles
// (x = M tile fastest, then N tile, then grid slice z) with two accumulators
// in tensor memory, so that a tile's epilogue overlaps the next tile's MMAs.
//   warp 0: allocates the 512 TMEM columns; one thread issues the TMA loads
//           of every tile's K blocks through the TC_STAGES ring;
//   warp 1: one thread waits for a free accumulator, issues the tile's MMAs
//           into it and commits them to tfull[buffer];
//   warps 2-5: the epilogue; warp w drains TMEM lanes 32 (w mod 4) .. +32
//           (its lane sub-partition), stores, and releases the accumulator
//           (tempty[buffer], one arrival per warp).
// Every wait is bounded; a wait that gives up raises the abort flag, which
// every other wait sees, and the kernel records PWH_ERR_TIMEOUT.
constexpr int TCP_THREADS = 192;
constexpr int TCP_TMEM_COLS = 512;

struct TcWork {
  int gm, gn, gz;  // M tiles, N tiles, grid slices
};

template <int MODE>
__global__ void __launch_bounds__(TCP_THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tma_a, const __grid_constant__ CUtensorMap tma_b,
              TcArgs args, TcWork wk) {
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + TC_STAGES * TC_STAGE_BYTES);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* tfull = empty + TC_STAGES;  // [2]
  uint64_t* tempty = tfull + 2;         // [2]
  uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles = wk.gm * wk.gn, items = tiles * wk.gz;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_slot)),
                 "r"(TCP_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  int issued = 0;  // producer: ring slots whose loads were started
  if (warp == 0 && lane == 0) {
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
      const int z = it / tiles, rem = it - z * tiles;
      const int m0 = (rem % wk.gm) * TC_BM, n0 = (rem / wk.gm) * TC_BN;
      int kb0, kb_end;
      tc_krange(args, z, kb0, kb_end);
      bool ok = true;
      for (int kb = kb0; kb < kb_end; ++kb) {
        const int s = issued % TC_STAGES;
        const uint32_t ph = ((issued / TC_STAGES) & 1) ^ 1;
        if (!mbar_wait(&empty[s], ph, abort_flag)) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        int xa, xb;
        if (args.oz) {
          const int t = kb / args.kb_seg, r = kb - t * args.kb_seg;
          xa = (args.oz_a[t] * args.kb_seg + r) * TC_BK;
          xb = (args.oz_b[t] * args.kb_seg + r) * TC_BK;
        } else {
          kb_coords(kb, args.kb_seg, xa, xb);
        }
        uint8_t* sa = smem + s * TC_STAGE_BYTES;
        mbar_expect_tx(&full[s], TC_STAGE_BYTES);
        tma_load_2d(sa, &tma_a, xa, m0, &full[s]);
        tma_load_2d(sa + TC_A_BYTES, &tma_b, xb, n0, &full[s]);
        ++issued;
      }
      if (!ok) break;
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_bf16(TC_BM, TC_BN);
    int used = 0, lj = 0;  // ring slots consumed, tiles of this CTA
    for (int it = blockIdx.x; it < items; it += gridDim.x, ++lj) {
      const int z = it / tiles;
      int kb0, kb_end;
      tc_krange(args, z, kb0, kb_end);
      const int nkb = max(0, kb_end - kb0);
      const int buf = lj & 1;
      if (!mbar_wait(&tempty[buf], ((lj >> 1) & 1) ^ 1, abort_flag)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t dst = tmem + (uint32_t)(buf * TC_BN);
      bool ok = true;
      for (int kb = 0; kb < nkb; ++kb, ++used) {
        const int s = used % TC_STAGES;
        if (!mbar_wait(&full[s], (used / TC_STAGES) & 1, abort_flag)) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = su32(smem + s * TC_STAGE_BYTES);
        const uint32_t b0 = a0 + TC_A_BYTES;
#pragma unroll
        for (int k = 0; k < TC_BK / 16; ++k)
          mma_bf16(dst, smem_desc(a0 + k * 32), smem_desc(b0 + k * 32), idesc,
                   (kb > 0 || k > 0) ? 1u : 0u);
        mma_commit(&empty[s]);
      }
      if (!ok) break;
      mma_commit(&tfull[buf]);  // arrives once every MMA issued so far has completed
    }
  } else if (warp >= 2) {
    const int sub = warp & 3;  // the TMEM lane sub-partition this warp may read
    const int row = sub * 32 + lane;
    int lj = 0;
    for (int it = blockIdx.x; it < items; it += gridDim.x, ++lj) {
      const int z = it / tiles, rem = it - z * tiles;
      const int m0 = (rem % wk.gm) * TC_BM, n0 = (rem / wk.gm) * TC_BN;
      int kb0, kb_end;
      tc_krange(args, z, kb0, kb_end);
      const int buf = lj & 1;
      if (!mbar_wait(&tfull[buf], (lj >> 1) & 1, abort_flag)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      if (kb_end > kb0) {
        const int m = m0 + row;
        for (int c0 = 0; c0 < TC_BN; c0 += 32) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(buf * TC_BN + c0), v);
          if (m < args.M) {
            if (MODE == 0) {
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const int n = n0 + c0 + j;
                if (n < args.N) args.part[((size_t)z * args.N + n) * args.M + m] = v[j];
              }
            } else {
              // the nonlocal term of band b at plane wave m, FP32 (the
              // z-forward FFT pass adds it into H psi)
#pragma unroll
              for (int j = 0; j < 32; j += 2) {
                const int b = (n0 + c0 + j) >> 1;
                if (b < args.nb) args.vnl[(size_t)b * args.ldv + m] = make_float2(v[j], v[j + 1]);
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
    }
  }
  __syncwarp();
  // producer: make sure every copy it started has landed before smem goes away
  if (warp == 0 && lane == 0) {
    for (int j = max(0, issued - TC_STAGES); j < issued; ++j)
      mbar_wait(&full[j % TC_STAGES], (j / TC_STAGES) & 1, nullptr);
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicExch(args.err, (int)PWH_ERR_TIMEOUT);
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TCP_TMEM_COLS)
                 : "memory");
  }
}

// Launches the persistent kernel over the gm x gn x gz grid of tiles and
// slices: one CTA per SM (fewer when there are fewer tiles).
template <int MODE>
static void tc_launch(const CUtensorMap& ma, const CUtensorMap& mb, const TcArgs& a, dim3 grid,
                      cudaStream_t st) {
  static int nsm = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 152;
    cudaFuncSetAttribute(k_tc_gemm<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    cudaFuncSetAttribute(k_tc_gemm<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  });
  TcWork wk{(int)grid.x, (int)grid.y, (int)grid.z};
  const int64_t items = (int64_t)grid.x * grid.y * grid.z;
  const int ctas = (int)std::max<int64_t>(1, std::min<int64_t>(items, nsm));
  k_tc_gemm<MODE><<<ctas, TCP_THREADS, TC_SMEM, st>>>(ma, mb, a, wk);
}

// ------------------------------------------------------- operand packing ----
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// A1[2p+c][G] (becp A operand) and A2[G][2p+c] (back-projection A operand),
// each [hi | lo] along K, from beta (internal order, FP64, column-major npw x P).
__global__ void k_pack_beta(const double2* __restrict__ beta, int64_t npw, int P,
                            __nv_bfloat16* __restrict__ A1, int64_t pitch1, int64_t seg1,
                            __nv_bfloat16* __restrict__ A2, int64_t pitch2, int64_t seg2) {
  int64_t tot = npw * P;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t g = t % npw, p = t / npw;
    double2 z = beta[t];
    __nv_bfloat16 rh, rl, ih, il;
    split_bf16((float)z.x, rh, rl);
    split_bf16((float)z.y, ih, il);
    __nv_bfloat16* r0 = A1 + (2 * p) * pitch1 + g;
    __nv_bfloat16* r1 = A1 + (2 * p + 1) * pitch1 + g;
    r0[0] = rh; r0[seg1] = rl;
    r1[0] = ih; r1[seg1] = il;
    __nv_bfloat16* q = A2 + g * pitch2 + 2 * p;
    q[0] = rh; q[1] = ih;
    q[seg2] = rl; q[seg2 + 1] = il;
  }
}

// B1[2b+c][G] from psi (FP64 complex, column-major npw x nb, leading dim ldp).
__global__ void k_pack_psi(const double2* __restrict__ psi, int64_t ldp, int64_t npw, int nb,
                           __nv_bfloat16* __restrict__ B1, int64_t pitch, int64_t seg) {
  int64_t tot = npw * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t g = t % npw, b = t / npw;
    double2 z = psi[b * ldp + g];
    __nv_bfloat16 rh, rl, ih, il;
    split_bf16((float)z.x, rh, rl);
    split_bf16((float)z.y, ih, il);
    __nv_bfloat16* r0 = B1 + (2 * b) * pitch + g;
    __nv_bfloat16* r1 = B1 + (2 * b + 1) * pitch + g;
    r0[0] = rh; r0[seg] = rl;
    r1[0] = ih; r1[seg] = il;
  }
}

// becp[p][b] (complex FP32, P x nb column-major) from the split-K partials of
// C1 (FP32, part[z][n][m], M = 2P, N = 2nb); diagonal D applied when given.
__global__ void k_becp_reduce(const float* __restrict__ part, int nsplit, int P, int nb,
                              const double* __restrict__ ddiag, float2* __restrict__ becp) {
  const int M = 2 * P, N = 2 * nb;
  int64_t tot = (int64_t)P * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    int p = (int)(t % P), b = (int)(t / P);
    float rr = 0, ri = 0, ir = 0, ii = 0;  // C[2p+x][2b+y]
    for (int z = 0; z < nsplit; ++z) {
      const float* pz = part + (size_t)z * M * N;
      rr += pz[(size_t)(2 * b) * M + 2 * p];
      ir += pz[(size_t)(2 * b) * M + 2 * p + 1];
      ri += pz[(size_t)(2 * b + 1) * M + 2 * p];
      ii += pz[(size_t)(2 * b + 1) * M + 2 * p + 1];
    }
    float re = rr + ii, im = ri - ir;
    if (ddiag) {
      float d = (float)ddiag[p];
      re *= d;
      im *= d;
    }
    becp[t] = make_float2(re, im);
  }
}

// B2[2b+c'][2p+c] ([hi | lo] along K) from becp' (complex FP32, P x nb).
__global__ void k_pack_becp(const float2* __restrict__ becp, int P, int nb,
                            __nv_bfloat16* __restrict__ B2, int64_t pitch, int64_t seg) {
  int64_t tot = (int64_t)P * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    int p = (int)(t % P), b = (int)(t / P);
    float2 z = becp[t];
    __nv_bfloat16 rh, rl, ih, il, nh, nl;
    split_bf16(z.x, rh, rl);
    split_bf16(z.y, ih, il);
    split_bf16(-z.y, nh, nl);
    __nv_bfloat16* r0 = B2 + (size_t)(2 * b) * pitch + 2 * p;
    __nv_bfloat16* r1 = B2 + (size_t)(2 * b + 1) * pitch + 2 * p;
    r0[0] = rh; r0[1] = nh; r0[seg] = rl; r0[seg + 1] = nl;
    r1[0] = ih; r1[1] = rh; r1[seg] = il; r1[seg + 1] = rl;
  }
}

__global__ void k_d_to_f32(const double2* __restrict__ src, int64_t n, float2* __restrict__ dst) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = make_float2((float)src[t].x, (float)src[t].y);
}

// ---------------------------------------------------------------- host -----
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  if (!fn) throw Error{PWH_ERR_CUDA, "cuTensorMapEncodeTiled unavailable"};
  return fn;
}

// 2D BF16 K-major tensor map: rows x cols (cols contiguous, pitch in elements),
// box 64 x box_rows, 128-byte swizzle, zero fill out of bounds.
static CUtensorMap make_map(const void* base, int64_t rows, int64_t cols, int64_t pitch,
                            int box_rows) {
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(pitch * 2)};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  if (((uintptr_t)base & 15) || ((pitch * 2) & 15))
    throw Error{PWH_ERR_ARG, "tensor map base or pitch not 16-byte aligned"};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                           strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error{PWH_ERR_CUDA, "cuTensorMapEncodeTiled failed"};
  return m;
}

static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Operand geometry for this system (K segments padded to whole 64-wide blocks).
struct TcGeom {
  int64_t seg1, pitch1;  // becp: K = npw
  int64_t seg2, pitch2;  // back-projection: K = 2P
};
static TcGeom geom(const System& s) {
  TcGeom g;
  g.seg1 = round_up(s.npw, TC_BK);
  g.pitch1 = 2 * g.seg1;
  g.seg2 = round_up(2 * (int64_t)s.nproj, TC_BK);
  g.pitch2 = 2 * g.seg2;
  return g;
}

void prepare_tc_projectors(System& s) {
  if (s.nproj == 0) return;
  TcGeom g = geom(s);
  const size_t n1 = (size_t)2 * s.nproj * g.pitch1, n2 = (size_t)s.npw * g.pitch2;
  PWH_CUDA(cudaMalloc(&s.d_beta_bf16, n1 * sizeof(__nv_bfloat16)));
  PWH_CUDA(cudaMalloc(&s.d_beta_bf16_t, n2 * sizeof(__nv_bfloat16)));
  PWH_CUDA(cudaMemsetAsync(s.d_beta_bf16, 0, n1 * sizeof(__nv_bfloat16), s.stream));
  PWH_CUDA(cudaMemsetAsync(s.d_beta_bf16_t, 0, n2 * sizeof(__nv_bfloat16), s.stream));
  k_pack_beta<<<2048, 256, 0, s.stream>>>(s.d_beta64, s.npw, s.nproj,
                                         (__nv_bfloat16*)s.d_beta_bf16, g.pitch1, g.seg1,
                                         (__nv_bfloat16*)s.d_beta_bf16_t, g.pitch2, g.seg2);
  PWH_LAUNCH_CHECK();
}

static void launch_tc(System& s, int mode, const CUtensorMap& ma, const CUtensorMap& mb, TcArgs a,
                      int gm, int gn, int gz, cudaStream_t st) {
  // algorithmic work: the real GEMM M x N x (terms x K) the launch performs
  const double kk = (double)a.terms * a.kb_seg * TC_BK;
  TimedScope ts(s, mode == 0 ? KF_TC_BECP : KF_TC_BACK, st, 2.0 * a.M * (double)a.N * kk,
                2.0 * ((double)a.M + a.N) * kk + (mode == 0 ? 4.0 * gz * (double)a.M * a.N
                                                            : 8.0 * a.M * (a.N / 2)));
  dim3 grid(gm, gn, gz);
  if (mode == 0)
    tc_launch<0>(ma, mb, a, grid, st);
  else
    tc_launch<1>(ma, mb, a, grid, st);
  PWH_LAUNCH_CHECK();
}

int* device_error_word(System& s);  // davidson.cu / hpsi.cu

void nonlocal_mixed(System& s, int nb, const double2* psi, int64_t ldp, float2* vnl, int64_t ldv,
                    cudaStream_t st, int terms) {
  if (s.nproj == 0 || nb <= 0) return;
  const int P = s.nproj;
  TcGeom g = geom(s);
  // ws_tc: B1 (2 cap x pitch1 bf16) | B2 (2 cap x pitch2 bf16) | becp, becp2, D32 (float2),
  // laid out for a band capacity; the K padding of B1/B2 is zeroed once per layout
  if (nb > s.tc_nb_cap || P != s.tc_P) {
    const int cap = std::max(nb, s.tc_nb_cap);
    const size_t need = ((size_t)2 * cap * (g.pitch1 + g.pitch2)) * sizeof(__nv_bfloat16) +
                        ((size_t)2 * P * cap + (size_t)P * P) * sizeof(float2) + 512;
    ensure(s.ws_tc, need);
    PWH_CUDA(cudaMemsetAsync(s.ws_tc.p, 0, s.ws_tc.n, st));
    s.tc_nb_cap = cap;
    s.tc_P = P;
  }
  const size_t b1 = (size_t)2 * s.tc_nb_cap * g.pitch1, b2 = (size_t)2 * s.tc_nb_cap * g.pitch2;
  __nv_bfloat16* B1 = (__nv_bfloat16*)s.ws_tc.p;
  __nv_bfloat16* B2 = B1 + b1;
  float2* becp = (float2*)(((uintptr_t)(B2 + b2) + 255) & ~(uintptr_t)255);
  float2* becp2 = becp + (size_t)P * nb;
  float2* d32 = becp2 + (size_t)P * nb;

  int gblk = (int)std::min<int64_t>(152 * 16, (s.npw * (int64_t)nb + 255) / 256);
  k_pack_psi<<<gblk, 256, 0, st>>>(psi, ldp, s.npw, nb, B1, g.pitch1, g.seg1);
  PWH_LAUNCH_CHECK();

  // ---- becp GEMM, split over K to fill the GPU: the split with the least
  // modelled time, waves of CTAs (one per SM at a time) times a CTA's share
  // of its tile's K on the tensor cores and about 2 us of set-up and
  // epilogue, plus the split-K partials written and read once more (nominal
  // rates: 2.25 PFLOP/s BF16, 7.9 TB/s)
  const int gm1 = (2 * P + TC_BM - 1) / TC_BM, gn1 = (2 * nb + TC_BN - 1) / TC_BN;
  const int kbs1 = (int)(g.seg1 / TC_BK);
  const int kbt1 = terms * kbs1;
  const int tiles1 = gm1 * gn1;
  const double tile_s = 2.0 * TC_BM * TC_BN * TC_BK * (double)kbt1 / (2.25e15 / 152);
  const double part_s = 2.0 * (2.0 * P) * (2.0 * nb) * sizeof(float) / 7.9e12;
  int split = 1;
  double best = 1e300;
  for (int sp = 1; sp <= std::min(64, kbt1); ++sp) {
    const double waves = (double)(((int64_t)tiles1 * sp + 151) / 152);
    const double t = waves * (tile_s / sp + 2e-6) + sp * part_s;
    if (t < best) {
      best = t;
      split = sp;
    }
  }
  int kper = (kbt1 + split - 1) / split;
  split = (kbt1 + kper - 1) / kper;  // every split gets >= 1 block
  ensure(s.ws_split, (size_t)split * 2 * P * 2 * nb * sizeof(float));
  CUtensorMap ma1 = make_map(s.d_beta_bf16, 2 * P, 2 * g.seg1, g.pitch1, TC_BM);
  CUtensorMap mb1 = make_map(B1, 2 * nb, 2 * g.seg1, g.pitch1, TC_BN);
  TcArgs a1{};
  a1.M = 2 * P; a1.N = 2 * nb; a1.kb_seg = kbs1; a1.terms = terms; a1.kb_per_split = kper;
  a1.part = (float*)s.ws_split.p; a1.err = device_error_word(s);
  launch_tc(s, 0, ma1, mb1, a1, gm1, gn1, split, st);
  int rb = (int)std::min<int64_t>(1024, ((int64_t)P * nb + 255) / 256);
  if (s.d_diag) {
    k_becp_reduce<<<rb, 256, 0, st>>>((const float*)s.ws_split.p, split, P, nb, s.d_ddiag, becp);
    PWH_LAUNCH_CHECK();
  } else {
    k_becp_reduce<<<rb, 256, 0, st>>>((const float*)s.ws_split.p, split, P, nb, nullptr, becp2);
    PWH_LAUNCH_CHECK();
    k_d_to_f32<<<64, 256, 0, st>>>(s.d_dfull, (int64_t)P * P, d32);
    PWH_LAUNCH_CHECK();
    const float2 one = make_float2(1, 0), zero = make_float2(0, 0);
    cgemm<float>(s, false, P, nb, P, one, d32, P, becp2, P, zero, becp, P, st);
  }
  k_pack_becp<<<rb, 256, 0, st>>>(becp, P, nb, B2, g.pitch2, g.seg2);
  PWH_LAUNCH_CHECK();

  // ---- back-projection GEMM into the FP32 buffer vnl
  const int gm2 = (int)((s.npw + TC_BM - 1) / TC_BM), gn2 = (2 * nb + TC_BN - 1) / TC_BN;
  const int kbs2 = (int)(g.seg2 / TC_BK);
  CUtensorMap ma2 = make_map(s.d_beta_bf16_t, s.npw, 2 * g.seg2, g.pitch2, TC_BM);
  CUtensorMap mb2 = make_map(B2, 2 * nb, 2 * g.seg2, g.pitch2, TC_BN);
  TcArgs a2{};
  a2.M = (int)s.npw; a2.N = 2 * nb; a2.kb_seg = kbs2; a2.terms = terms;
  a2.kb_per_split = terms * kbs2; a2.vnl = vnl; a2.ldv = ldv; a2.nb = nb;
  a2.err = device_error_word(s);
  launch_tc(s, 1, ma2, mb2, a2, gm2, gn2, 1, st);
}


// ------------------------------------ FP64-equivalent complex GEMM (slices) ----
// C = alpha op(A) B + beta C for FP64 (complex128) operands on the BF16 tensor
// cores, accurate to about FP64 rounding: the error-free splitting of Ozaki et
// al. (products of integer slices summed exactly).  Each real row r of an
// operand (after the complex interleaving of the projector GEMM above) gets
// the exponent e_r with max|x_r| < 2^e_r and is written as
//     x = 2^e_r sum_{s < OZ_S} a_s 2^(-6 - 7 s),   a_s integers, |a_s| <= 64,
// which BF16 holds exactly (balanced base-128 digits of the row-scaled value
// as an integer).  A product a_s b_t is at most 2^12 and a sum of 4096 of
// them at most 2^24, so every FP32 partial of a 4096-wide K chunk is an exact
// integer (base-128 digits take one slice more than base-256 ones, 36 pairs
// instead of 28, and write a third of the partials).  The partials of the
// pairs with s + t <= OZ_G are summed in int64 by weight 2^(-7(s+t)) and
// scaled once in FP64.  Dropped terms and slice truncation are below 2^-52 of
// max|a| max|b| per elementary product.
constexpr int OZ_S = 8;
constexpr int OZ_G = OZ_S - 1;
constexpr int OZ_PAIRS = (OZ_S * (OZ_S + 1)) / 2;  // pairs with s + t <= OZ_G
constexpr int OZ_CHUNK_KB = 64;                    // 64-wide K blocks per exact partial
static_assert(OZ_PAIRS <= 64, "pair table");
__constant__ unsigned char c_oz_g[64];            // s + t of pair p

// Slicing works on the IEEE bit patterns with integer arithmetic only (the
// FP64 pipe of this GPU would make it the slowest step).  |x| as an unsigned
// integer orders like |x|, so row maxima are integer maxima of these keys.
__device__ __forceinline__ unsigned long long oz_key(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
// exponent e with |x| < 2^e for the largest key of a row (0 for a zero row)
__device__ __forceinline__ int oz_exp_of_key(unsigned long long k) {
  if (k == 0) return 0;
  const int eb = (int)(k >> 52);
  return eb ? eb - 1022 : -1021;  // frexp exponent; subnormals lie below 2^-1022
}
// The OZ_S balanced base-128 digits of X = round(x 2^(55 - e)), |X| < 2^55:
// x = 2^e sum_s a_s 2^(-6 - 7 s) up to 2^(e - 56), |a_s| <= 64, as BF16.
__device__ __forceinline__ void oz_split(double x, int e, __nv_bfloat16* a) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int eb = (int)((bits >> 52) & 0x7ff);
  const unsigned long long m = (bits & 0xfffffffffffffull) | (eb ? (1ull << 52) : 0ull);
  const int sh = (eb ? eb : 1) - 1075 + 55 - e;  // X = m 2^sh
  long long X;
  if (sh >= 0) X = (long long)(m << sh);
  else if (sh > -64) X = (long long)((m + (1ull << (-sh - 1))) >> (-sh));
  else X = 0;
  if (bits >> 63) X = -X;
#pragma unroll
  for (int s = OZ_S - 1; s > 0; --s) {
    const int d = (int)((X + 64) & 127) - 64;
    a[s] = __int2bfloat16_rn(d);
    X = (X - d) >> 7;
  }
  a[0] = __int2bfloat16_rn((int)X);
}

// Exponents of the rows 2j (real parts) and 2j+1 (imaginary parts) of the
// interleaved operand whose row pair j is column j of X (K x J, ld): one block
// per column.
__global__ void k_oz_colexp(const double2* __restrict__ X, int64_t ld, int K, int* __restrict__ ex) {
  __shared__ unsigned long long red[2][32];
  const int j = blockIdx.x;
  unsigned long long mr = 0, mi = 0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const double2 v = X[(size_t)j * ld + k];
    mr = max(mr, oz_key(v.x));
    mi = max(mi, oz_key(v.y));
  }
  for (int o = 16; o > 0; o >>= 1) {
    mr = max(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    mi = max(mi, __shfl_xor_sync(0xffffffffu, mi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = mr;
    red[1][threadIdx.x >> 5] = mi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      mr = max(mr, red[0][w]);
      mi = max(mi, red[1][w]);
    }
    ex[2 * j] = oz_exp_of_key(mr);
    ex[2 * j + 1] = oz_exp_of_key(mi);
  }
}
// Slices of that operand: row 2j+c, segment s holds a_s of (Re, Im) X[k][j]
// at column s seg + k (zero for K <= k < seg).
__global__ void k_oz_slice_cols(const double2* __restrict__ X, int64_t ld, int K, int seg,
                                const int* __restrict__ ex, __nv_bfloat16* __restrict__ out,
                                int64_t pitch) {
  const int j = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= seg) return;
  const double2 v = k < K ? X[(size_t)j * ld + k] : make_double2(0.0, 0.0);
  __nv_bfloat16 ar[OZ_S], ai[OZ_S];
  oz_split(v.x, ex[2 * j], ar);
  oz_split(v.y, ex[2 * j + 1], ai);
  __nv_bfloat16* r0 = out + (size_t)(2 * j) * pitch + k;
  __nv_bfloat16* r1 = r0 + pitch;
#pragma unroll
  for (int s = 0; s < OZ_S; ++s) {
    r0[(size_t)s * seg] = ar[s];
    r1[(size_t)s * seg] = ai[s];
  }
}

// Exponent of row m of the operand A2[m][2k+c] = (Re, Im) A[m][k] (A: M x K,
// column-major, ld): one thread per row.
__global__ void k_oz_rowexp(const double2* __restrict__ A, int64_t ld, int M, int K,
                            int* __restrict__ ex) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  unsigned long long mx = 0;
  for (int k = 0; k < K; ++k) {
    const double2 v = A[(size_t)k * ld + m];
    mx = max(mx, max(oz_key(v.x), oz_key(v.y)));
  }
  ex[m] = oz_exp_of_key(mx);
}
// Slices of A2: row m, segment s, column 2k+c (zero for 2K <= 2k+c < seg);
// 32 x 32 tiles transposed through shared memory.
__global__ void k_oz_slice_rows(const double2* __restrict__ A, int64_t ld, int M, int K, int seg,
                                const int* __restrict__ ex, __nv_bfloat16* __restrict__ out,
                                int64_t pitch) {
  __shared__ double2 tile[32][33];
  const int m0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int t = threadIdx.x; t < 1024; t += blockDim.x) {
    const int mm = t & 31, kk = t >> 5;
    const int m = m0 + mm, k = k0 + kk;
    tile[kk][mm] = (m < M && k < K) ? A[(size_t)k * ld + m] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 1024; t += blockDim.x) {
    const int kk = t & 31, mm = t >> 5;
    const int m = m0 + mm, k = k0 + kk;
    if (m >= M || 2 * k >= seg) continue;
    const double2 v = tile[kk][mm];
    const int e = ex[m];
    __nv_bfloat16 ar[OZ_S], ai[OZ_S];
    oz_split(v.x, e, ar);
    oz_split(v.y, e, ai);
    __nv_bfloat16* r = out + (size_t)m * pitch + 2 * k;
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      __nv_bfloat162 p;
      p.x = ar[s];
      p.y = ai[s];
      *(__nv_bfloat162*)(r + (size_t)s * seg) = p;
    }
  }
}

// B operand of the non-conjugated product: rows 2n, 2n+1 of
//     B2[2n][2k] = Re, B2[2n][2k+1] = -Im, B2[2n+1][2k] = Im, B2[2n+1][2k+1] = Re
// of B[k][n] (B: K x N, column-major, ld), both rows with the exponent of
// max(|Re|, |Im|) over column n: one block per column.
__global__ void k_oz_colexp_b2(const double2* __restrict__ B, int64_t ld, int K,
                               int* __restrict__ ex) {
  __shared__ unsigned long long red[32];
  const int n = blockIdx.x;
  unsigned long long mx = 0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const double2 v = B[(size_t)n * ld + k];
    mx = max(mx, max(oz_key(v.x), oz_key(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = max(mx, red[w]);
    ex[2 * n] = ex[2 * n + 1] = oz_exp_of_key(mx);
  }
}
__global__ void k_oz_slice_b2(const double2* __restrict__ B, int64_t ld, int K, int seg,
                              const int* __restrict__ ex, __nv_bfloat16* __restrict__ out,
                              int64_t pitch) {
  const int n = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * k >= seg) return;
  const double2 v = k < K ? B[(size_t)n * ld + k] : make_double2(0.0, 0.0);
  const int e = ex[2 * n];
  __nv_bfloat16 ar[OZ_S], ai[OZ_S];
  oz_split(v.x, e, ar);
  oz_split(v.y, e, ai);
  __nv_bfloat16* r0 = out + (size_t)(2 * n) * pitch + 2 * k;
  __nv_bfloat16* r1 = r0 + pitch;
#pragma unroll
  for (int s = 0; s < OZ_S; ++s) {
    __nv_bfloat162 p0, p1;
    p0.x = ar[s];
    p0.y = __hneg(ai[s]);
    p1.x = ai[s];
    p1.y = ar[s];
    *(__nv_bfloat162*)(r0 + (size_t)s * seg) = p0;
    *(__nv_bfloat162*)(r1 + (size_t)s * seg) = p1;
  }
}

// Exact accumulation of the integer partials of one real output: weights
// 2^(-7g) folded into hi (g <= 3) and lo (g >= 4); value
// 2^(e - 12) (hi 2^-21 + lo 2^-(7 OZ_G)).  At 161,235-wide K (40 chunks) both
// stay below 2^53.
struct OzAcc {
  long long hi = 0, lo = 0;
  // i: a sum of exact integer partials (each |v| <= 2^24) of weight 2^(-7g)
  __device__ __forceinline__ void add_int(long long i, int g) {
    if (g <= 3) hi += i * (1ll << (7 * (3 - g)));
    else lo += i * (1ll << (7 * (OZ_G - g)));
  }
  __device__ __forceinline__ double value(int e) const {
    return ldexp((double)hi, e - 12 - 21) + ldexp((double)lo, e - 12 - 7 * OZ_G);
  }
};

// op(A) = A^H: complex (m, n) from the four real products of rows 2m, 2m+1 and
// columns 2n, 2n+1 (Re = C[2m][2n] + C[2m+1][2n+1], Im = C[2m][2n+1] -
// C[2m+1][2n]); part[z][n'][m'] with M' = 2M, N' = 2N, z = chunk * pairs + pair.
__global__ void k_oz_reduce_cj(const float* __restrict__ part, int nz, int nchunk, int M, int N,
                               const int* __restrict__ exa, const int* __restrict__ exb,
                               const double* __restrict__ rowscale, double2 alpha, double2 beta,
                               double2* __restrict__ C, int64_t ldc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)M * N) return;
  const int m = (int)(t % M), n = (int)(t / M);
  const int64_t Mr = 2 * (int64_t)M, plane = Mr * 2 * (int64_t)N;
  OzAcc q00, q10, q01, q11;
  const float* p0 = part + (size_t)(2 * n) * Mr + 2 * m;      // (2m,2n), (2m+1,2n)
  const float* p1 = part + (size_t)(2 * n + 1) * Mr + 2 * m;  // (2m,2n+1), (2m+1,2n+1)
  const int npair = nz / nchunk;
  for (int pr = 0; pr < npair; ++pr) {
    const int g = c_oz_g[pr];
    // the chunks of one pair share the weight: integer sums first, four
    // partials in flight
    long long s00 = 0, s10 = 0, s01 = 0, s11 = 0;
    int c = 0;
    for (; c + 3 < nchunk; c += 4) {
      float2 a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const size_t z = (size_t)(c + u) * npair + pr;
        a[u] = *(const float2*)(p0 + z * plane);
        b[u] = *(const float2*)(p1 + z * plane);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        s00 += __float2int_rn(a[u].x);
        s10 += __float2int_rn(a[u].y);
        s01 += __float2int_rn(b[u].x);
        s11 += __float2int_rn(b[u].y);
      }
    }
    for (; c < nchunk; ++c) {
      const size_t z = (size_t)c * npair + pr;
      const float2 a = *(const float2*)(p0 + z * plane), b = *(const float2*)(p1 + z * plane);
      s00 += __float2int_rn(a.x);
      s10 += __float2int_rn(a.y);
      s01 += __float2int_rn(b.x);
      s11 += __float2int_rn(b.y);
    }
    q00.add_int(s00, g);
    q10.add_int(s10, g);
    q01.add_int(s01, g);
    q11.add_int(s11, g);
  }
  const int ea0 = exa[2 * m], ea1 = exa[2 * m + 1], eb0 = exb[2 * n], eb1 = exb[2 * n + 1];
  double re = q00.value(ea0 + eb0) + q11.value(ea1 + eb1);
  double im = q01.value(ea0 + eb1) - q10.value(ea1 + eb0);
  if (rowscale) {
    re *= rowscale[m];
    im *= rowscale[m];
  }
  double2 r = make_double2(alpha.x * re - alpha.y * im, alpha.x * im + alpha.y * re);
  if (beta.x != 0.0 || beta.y != 0.0) {
    const double2 c = C[(size_t)n * ldc + m];
    r.x += beta.x * c.x - beta.y * c.y;
    r.y += beta.x * c.y + beta.y * c.x;
  }
  C[(size_t)n * ldc + m] = r;
}

// op(A) = A: complex (m, n) = (C2[m][2n], C2[m][2n+1]); part[z][n'][m'] with
// M' = M, N' = 2N.
__global__ void k_oz_reduce_nn(const float* __restrict__ part, int nz, int nchunk, int M, int N,
                               const int* __restrict__ exa, const int* __restrict__ exb,
                               const double* __restrict__ rowscale, double2 alpha, double2 beta,
                               double2* __restrict__ C, int64_t ldc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)M * N) return;
  const int m = (int)(t % M), n = (int)(t / M);
  const int64_t plane = (int64_t)M * 2 * N;
  OzAcc qr, qi;
  const float* p0 = part + (size_t)(2 * n) * M + m;
  const float* p1 = p0 + M;
  const int npair = nz / nchunk;
  if (nchunk == 1) {
    // one chunk: every pair's partial in flight together
#pragma unroll 9
    for (int pr = 0; pr < OZ_PAIRS; ++pr) {
      qr.add_int(__float2int_rn(p0[(size_t)pr * plane]), c_oz_g[pr]);
      qi.add_int(__float2int_rn(p1[(size_t)pr * plane]), c_oz_g[pr]);
    }
  } else {
    for (int pr = 0; pr < npair; ++pr) {
      long long sr = 0, si = 0;
      for (int c = 0; c < nchunk; ++c) {
        const size_t z = (size_t)c * npair + pr;
        sr += __float2int_rn(p0[z * plane]);
        si += __float2int_rn(p1[z * plane]);
      }
      qr.add_int(sr, c_oz_g[pr]);
      qi.add_int(si, c_oz_g[pr]);
    }
  }
  const int e = exa[m] + exb[2 * n];
  double re = qr.value(e), im = qi.value(e);
  if (rowscale) {
    re *= rowscale[m];
    im *= rowscale[m];
  }
  double2 r = make_double2(alpha.x * re - alpha.y * im, alpha.x * im + alpha.y * re);
  if (beta.x != 0.0 || beta.y != 0.0) {
    const double2 c = C[(size_t)n * ldc + m];
    r.x += beta.x * c.x - beta.y * c.y;
    r.y += beta.x * c.y + beta.y * c.x;
  }
  C[(size_t)n * ldc + m] = r;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Geometry and workspace of one sliced product.
struct OzGeom {
  int64_t Mr, Nr, seg, pitch;
  int kb_seg, kbps, nchunk, nz;
  size_t bytes_a, bytes_b, bytes_e, bytes_p;
  size_t total() const { return bytes_a + bytes_b + bytes_e + bytes_p; }
};
static OzGeom oz_geom(bool conjA, int M, int N, int K) {
  OzGeom g;
  // real GEMM geometry: C' (Mr x Nr) = A' (Mr x Kr) B'^T, both K-major
  g.Mr = conjA ? 2 * (int64_t)M : M;
  g.Nr = 2 * (int64_t)N;
  const int64_t Kr = conjA ? K : 2 * (int64_t)K;
  g.seg = round_up(std::max<int64_t>(Kr, 1), TC_BK);
  g.kb_seg = (int)(g.seg / TC_BK);
  // K blocks per exact partial: at most OZ_CHUNK_KB (4096 wide) and dividing
  // kb_seg; pad the segment to whole chunks when that costs little, else take
  // a divisor of at least half a chunk
  g.kbps = g.kb_seg;
  if (g.kb_seg > OZ_CHUNK_KB) {
    const int padc = (g.kb_seg + OZ_CHUNK_KB - 1) / OZ_CHUNK_KB * OZ_CHUNK_KB;
    g.kbps = 0;
    if ((padc - g.kb_seg) * 16 > g.kb_seg)
      for (int d = OZ_CHUNK_KB; d >= OZ_CHUNK_KB / 2 && !g.kbps; --d)
        if (g.kb_seg % d == 0) g.kbps = d;
    if (!g.kbps) {
      g.kb_seg = padc;
      g.seg = (int64_t)g.kb_seg * TC_BK;
      g.kbps = OZ_CHUNK_KB;
    }
  }
  g.nchunk = g.kb_seg / g.kbps;
  g.nz = OZ_PAIRS * g.nchunk;
  g.pitch = OZ_S * g.seg;
  g.bytes_a = align256((size_t)g.Mr * g.pitch * 2);
  g.bytes_b = align256((size_t)g.Nr * g.pitch * 2);
  g.bytes_e = align256((size_t)(g.Mr + g.Nr) * sizeof(int));
  g.bytes_p = (size_t)g.nz * g.Mr * g.Nr * sizeof(float);
  return g;
}

// The exact partials (OZ_PAIRS per K chunk, FP32, of the whole real output) are
// bounded.  A product over many chunks first runs as K segments of whole
// chunks, each added into C in FP64 (one more rounding per segment, no
// operand sliced twice); a segment that still does not fit runs as pieces of
// its larger output dimension, which give the same bits as the whole segment
// (the exponents belong to single rows of op(A) and single columns of B).
constexpr size_t kOzPartCap = (size_t)4 << 30;
constexpr int kOzSegChunks = 8;

struct OzSplit {
  int kseg;      // complex K per segment
  bool split_m;  // pieces of M (else of N)
  int piece;     // rows or columns per piece
};
static OzSplit oz_split_of(bool conjA, int M, int N, int K) {
  OzSplit sp{K, M >= N, M >= N ? M : N};
  // at most kOzSegChunks 4096-wide real chunks a segment: the slices are
  // stored [row][slice * seg + k], so the row pitch grows with the segment
  // and one chunk's tiles spread over as many memory pages as there are rows
  // (a 544 x 544 x 161,235 A^H B product ran its 25-chunk first segment at
  // 0.57 ms a chunk and its 15-chunk second one at 0.36 ms)
  const int kmax = (conjA ? 64 : 32) * OZ_CHUNK_KB * kOzSegChunks;
  if (K > kmax) sp.kseg = kmax;
  const OzGeom g = oz_geom(conjA, M, N, sp.kseg);
  if (g.bytes_p <= kOzPartCap) return sp;
  const size_t per_chunk = g.bytes_p / (size_t)g.nchunk;
  if (g.nchunk > 1) {
    // whole 4096-wide real chunks per segment (4096 complex K for A^H B,
    // 2048 for A B, whose real K is 2K)
    const int64_t c = std::max<int64_t>(1, (int64_t)(kOzPartCap / per_chunk));
    const int64_t kc = conjA ? 64 * OZ_CHUNK_KB : 32 * OZ_CHUNK_KB;
    if (c < g.nchunk) sp.kseg = (int)std::min<int64_t>(sp.kseg, c * kc);
  }
  const OzGeom gs = oz_geom(conjA, M, N, sp.kseg);
  if (gs.bytes_p <= kOzPartCap) return sp;
  const size_t per = gs.bytes_p / (size_t)sp.piece;  // partial bytes per row or column
  const int64_t fit = (int64_t)(kOzPartCap / per) / 64 * 64;
  sp.piece = (int)std::max<int64_t>(64, std::min<int64_t>(fit, sp.piece));
  return sp;
}

void oz_reserve(System& s, bool conjA, int M, int N, int K) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  const OzSplit sp = oz_split_of(conjA, M, N, K);
  ensure(s.ws_oz, oz_geom(conjA, sp.split_m ? std::min(sp.piece, M) : M,
                          sp.split_m ? N : std::min(sp.piece, N), sp.kseg)
                      .total());
}

static void oz_gemm_piece(System& s, bool conjA, int M, int N, int K, double2 alpha,
                          const double2* A, int64_t lda, const double2* B, int64_t ldb,
                          double2 beta, double2* C, int64_t ldc, cudaStream_t st,
                          const double* rowscale);

void oz_gemm(System& s, bool conjA, int M, int N, int K, double2 alpha, const double2* A,
             int64_t lda, const double2* B, int64_t ldb, double2 beta, double2* C, int64_t ldc,
             cudaStream_t st, const double* rowscale) {
  if (M <= 0 || N <= 0) return;
  const OzSplit sp = oz_split_of(conjA, M, N, K);
  for (int k0 = 0; k0 == 0 || k0 < K; k0 += sp.kseg) {
    const int kk = std::min(sp.kseg, K - k0);
    // K rows k0.. of B and of A (A^H), or K columns k0.. of A
    const double2* Ak = A + (conjA ? (int64_t)k0 : (int64_t)k0 * lda);
    const double2* Bk = B + k0;
    const double2 bk = k0 == 0 ? beta : make_double2(1, 0);
    if (sp.split_m) {
      // rows m0.. of C: columns m0.. of A (A^H) or rows m0.. of A
      for (int m0 = 0; m0 < M; m0 += sp.piece)
        oz_gemm_piece(s, conjA, std::min(sp.piece, M - m0), N, kk, alpha,
                      Ak + (conjA ? (int64_t)m0 * lda : (int64_t)m0), lda, Bk, ldb, bk, C + m0,
                      ldc, st, rowscale ? rowscale + m0 : nullptr);
    } else {
      for (int n0 = 0; n0 < N; n0 += sp.piece)
        oz_gemm_piece(s, conjA, M, std::min(sp.piece, N - n0), kk, alpha, Ak, lda,
                      Bk + (int64_t)n0 * ldb, ldb, bk, C + (int64_t)n0 * ldc, ldc, st, rowscale);
    }
  }
}

static void oz_gemm_piece(System& s, bool conjA, int M, int N, int K, double2 alpha,
                          const double2* A, int64_t lda, const double2* B, int64_t ldb,
                          double2 beta, double2* C, int64_t ldc, cudaStream_t st,
                          const double* rowscale) {
  static std::once_flag once;
  static unsigned char pa[64], pb[64];
  std::call_once(once, [] {
    unsigned char g[64] = {};
    // pairs by A slice, then B slice: consecutive grid slices share an A
    // slice, so one K chunk needs one A slice and its B slices in L2 at a time
    int p = 0;
    for (int sa = 0; sa <= OZ_G; ++sa)
      for (int sb = 0; sa + sb <= OZ_G; ++sb) {
        pa[p] = (unsigned char)sa;
        pb[p] = (unsigned char)sb;
        g[p] = (unsigned char)(sa + sb);
        ++p;
      }
    cudaMemcpyToSymbol(c_oz_g, g, sizeof(g));
    cudaFuncSetAttribute(k_tc_gemm<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  });
  const OzGeom gg = oz_geom(conjA, M, N, K);
  const int64_t Mr = gg.Mr, Nr = gg.Nr, seg = gg.seg;
  const int kb_seg = gg.kb_seg, kbps = gg.kbps, nchunk = gg.nchunk, nz = gg.nz;
  const int64_t pitch = gg.pitch;
  const size_t bytes_a = gg.bytes_a, bytes_b = gg.bytes_b, bytes_e = gg.bytes_e;
  ensure(s.ws_oz, gg.total());
  char* base = s.ws_oz.p;
  __nv_bfloat16* pA = (__nv_bfloat16*)base;
  __nv_bfloat16* pB = (__nv_bfloat16*)(base + bytes_a);
  int* exa = (int*)(base + bytes_a + bytes_b);
  int* exb = exa + Mr;
  float* part = (float*)(base + bytes_a + bytes_b + bytes_e);

  // timed as its own family: the work is the real BF16 tensor-core GEMM of
  // all slice pairs (2 Mr Nr Kr per pair)
  TimedScope ts(s, KF_GEMM_OZ, st, 2.0 * OZ_PAIRS * (double)Mr * Nr * (double)seg,
                2.0 * OZ_PAIRS * ((double)Mr + Nr) * seg + 8.0 * nz * (double)Mr * Nr);
  // slices of op(A) and B
  if (conjA) {
    k_oz_colexp<<<M, 256, 0, st>>>(A, lda, K, exa);
    PWH_LAUNCH_CHECK();
    k_oz_slice_cols<<<dim3((unsigned)((seg + 255) / 256), M), 256, 0, st>>>(A, lda, K, (int)seg, exa,
                                                                            pA, pitch);
    PWH_LAUNCH_CHECK();
    k_oz_colexp<<<N, 256, 0, st>>>(B, ldb, K, exb);
    PWH_LAUNCH_CHECK();
    k_oz_slice_cols<<<dim3((unsigned)((seg + 255) / 256), N), 256, 0, st>>>(B, ldb, K, (int)seg, exb,
                                                                            pB, pitch);
    PWH_LAUNCH_CHECK();
  } else {
    k_oz_rowexp<<<(M + 255) / 256, 256, 0, st>>>(A, lda, M, K, exa);
    PWH_LAUNCH_CHECK();
    k_oz_slice_rows<<<dim3((M + 31) / 32, (unsigned)((seg / 2 + 31) / 32)), 256, 0, st>>>(
        A, lda, M, K, (int)seg, exa, pA, pitch);
    PWH_LAUNCH_CHECK();
    k_oz_colexp_b2<<<N, 256, 0, st>>>(B, ldb, K, exb);
    PWH_LAUNCH_CHECK();
    k_oz_slice_b2<<<dim3((unsigned)((seg / 2 + 255) / 256), N), 256, 0, st>>>(B, ldb, K, (int)seg,
                                                                              exb, pB, pitch);
    PWH_LAUNCH_CHECK();
  }
  // every slice pair, every K chunk: exact FP32 partials on the tensor cores
  CUtensorMap ma = make_map(pA, Mr, pitch, pitch, TC_BM);
  CUtensorMap mb = make_map(pB, Nr, pitch, pitch, TC_BN);
  TcArgs a{};
  a.M = (int)Mr;
  a.N = (int)Nr;
  a.kb_seg = kb_seg;
  a.terms = OZ_PAIRS;
  a.kb_per_split = kbps;
  a.part = part;
  a.err = device_error_word(s);
  a.oz = 1;
  for (int p = 0; p < OZ_PAIRS; ++p) {
    a.oz_a[p] = pa[p];
    a.oz_b[p] = pb[p];
  }
  dim3 grid((unsigned)((Mr + TC_BM - 1) / TC_BM), (unsigned)((Nr + TC_BN - 1) / TC_BN), nz);
  tc_launch<0>(ma, mb, a, grid, st);
  PWH_LAUNCH_CHECK();
  const int64_t tot = (int64_t)M * N;
  if (conjA)
    k_oz_reduce_cj<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(part, nz, nchunk, M, N, exa, exb,
                                                                  rowscale, alpha, beta, C, ldc);
  else
    k_oz_reduce_nn<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(part, nz, nchunk, M, N, exa, exb,
                                                                  rowscale, alpha, beta, C, ldc);
  PWH_LAUNCH_CHECK();
}

// ------------------------------------- FP32-equivalent GEMM (3 BF16 slices) --
// Each real operand value, rounded to FP32, is the exact sum of three BF16
// values x = x0 + x1 + x2 (x0 = bf16(x), x1 = bf16(x - x0), x2 = x - x0 - x1:
// 8 significant bits each, 24 in all, every slice with its own exponent).  The
// six products with s + t <= 2 run as one BF16 GEMM over the concatenated K
// segments, accumulating in FP32 tensor memory; the three dropped products are
// below 2^-26 of |a b|.  Split-K partials are summed in FP64.
constexpr int X3_S = 3, X3_TERMS = 6;

// NSL = 3: the FP32 value as three BF16 slices (exact); NSL = 2: its two
// leading slices, the second rounded (about 16 significant bits).
template <int NSL>
__device__ __forceinline__ void x3_split(double x, __nv_bfloat16* a) {
  const float f = d2f_rn(x);
  a[0] = __float2bfloat16_rn(f);
  const float r1 = f - __bfloat162float(a[0]);  // exact: at most 16 significant bits
  a[1] = __float2bfloat16_rn(r1);
  if constexpr (NSL == 3) a[2] = __float2bfloat16_rn(r1 - __bfloat162float(a[1]));  // exact remainder
}

// Rows 2j (real parts) and 2j+1 (imaginary parts) of the interleaved operand
// whose row pair j is column j of X (K x J, ld): segment s holds slice s at
// column s seg + k (zero for K <= k < seg); two K positions per thread.
template <int NSL>
__global__ void k_x3_slice_cols(const double2* __restrict__ X, int64_t ld, int K, int seg,
                                __nv_bfloat16* __restrict__ out, int64_t pitch) {
  const int j = blockIdx.y;
  const int k = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (k >= seg) return;
  const double2* x = X + (size_t)j * ld;
  const double2 v0 = k < K ? x[k] : make_double2(0.0, 0.0);
  const double2 v1 = k + 1 < K ? x[k + 1] : make_double2(0.0, 0.0);
  __nv_bfloat16 r0[NSL], i0[NSL], r1[NSL], i1[NSL];
  x3_split<NSL>(v0.x, r0);
  x3_split<NSL>(v0.y, i0);
  x3_split<NSL>(v1.x, r1);
  x3_split<NSL>(v1.y, i1);
  __nv_bfloat16* o0 = out + (size_t)(2 * j) * pitch + k;
  __nv_bfloat16* o1 = o0 + pitch;
#pragma unroll
  for (int t = 0; t < NSL; ++t) {
    __nv_bfloat162 p, q;
    p.x = r0[t];
    p.y = r1[t];
    q.x = i0[t];
    q.y = i1[t];
    *(__nv_bfloat162*)(o0 + (size_t)t * seg) = p;
    *(__nv_bfloat162*)(o1 + (size_t)t * seg) = q;
  }
}

// A2[m][s seg + 2k + c] = slice s of (Re, Im) A[m][k] (A: M x K column-major,
// zero for 2K <= 2k + c < seg); 32 x 32 tiles transposed through shared memory.
template <int NSL>
__global__ void k_x3_slice_rows(const double2* __restrict__ A, int64_t ld, int M, int K, int seg,
                                __nv_bfloat16* __restrict__ out, int64_t pitch) {
  __shared__ double2 tile[32][33];
  const int m0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int t = threadIdx.x; t < 1024; t += blockDim.x) {
    const int mm = t & 31, kk = t >> 5;
    const int m = m0 + mm, k = k0 + kk;
    tile[kk][mm] = (m < M && k < K) ? A[(size_t)k * ld + m] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 1024; t += blockDim.x) {
    const int kk = t & 31, mm = t >> 5;
    const int m = m0 + mm, k = k0 + kk;
    if (m >= M || 2 * k >= seg) continue;
    const double2 v = tile[kk][mm];
    __nv_bfloat16 ar[NSL], ai[NSL];
    x3_split<NSL>(v.x, ar);
    x3_split<NSL>(v.y, ai);
    __nv_bfloat16* r = out + (size_t)m * pitch + 2 * k;
#pragma unroll
    for (int s = 0; s < NSL; ++s) {
      __nv_bfloat162 p;
      p.x = ar[s];
      p.y = ai[s];
      *(__nv_bfloat162*)(r + (size_t)s * seg) = p;
    }
  }
}

// B operand of the non-conjugated product, rows 2n and 2n+1:
//     B2[2n][2k] = Re, B2[2n][2k+1] = -Im, B2[2n+1][2k] = Im, B2[2n+1][2k+1] = Re
// of B[k][n] (B: K x N column-major), each value as its three slices.
template <int NSL>
__global__ void k_x3_slice_b2(const double2* __restrict__ B, int64_t ld, int K, int seg,
                              __nv_bfloat16* __restrict__ out, int64_t pitch) {
  const int n = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * k >= seg) return;
  const double2 v = k < K ? B[(size_t)n * ld + k] : make_double2(0.0, 0.0);
  __nv_bfloat16 ar[NSL], ai[NSL];
  x3_split<NSL>(v.x, ar);
  x3_split<NSL>(v.y, ai);
  __nv_bfloat16* r0 = out + (size_t)(2 * n) * pitch + 2 * k;
  __nv_bfloat16* r1 = r0 + pitch;
#pragma unroll
  for (int s = 0; s < NSL; ++s) {
    __nv_bfloat162 p0, p1;
    p0.x = ar[s];
    p0.y = __hneg(ai[s]);
    p1.x = ai[s];
    p1.y = ar[s];
    *(__nv_bfloat162*)(r0 + (size_t)s * seg) = p0;
    *(__nv_bfloat162*)(r1 + (size_t)s * seg) = p1;
  }
}

// Epilogue of the reducers: C = alpha v + beta C with v the FP32 sum of the
// partials.  beta = 0 or 1 with a real FP32 alpha (every product of the
// eigensolver) takes FP32 arithmetic and integer format conversions; other
// coefficients take FP64.
struct X3Out {
  double2 alpha, beta;
  float af;  // alpha.x in FP32
  int mode;  // 0: beta = 0, real alpha; 1: beta = 1, real alpha; 2: general
};
__device__ __forceinline__ void x3_store(const X3Out& o, float re, float im, double2* c) {
  if (o.mode == 0) {
    *c = f2d(make_float2(o.af * re, o.af * im));
  } else if (o.mode == 1) {
    const double2 v = f2d(make_float2(o.af * re, o.af * im));
    const double2 c0 = *c;
    *c = make_double2(c0.x + v.x, c0.y + v.y);
  } else {
    const double2 v = f2d(make_float2(re, im));
    double2 r = make_double2(o.alpha.x * v.x - o.alpha.y * v.y, o.alpha.x * v.y + o.alpha.y * v.x);
    if (o.beta.x != 0.0 || o.beta.y != 0.0) {
      const double2 c0 = *c;
      r.x += o.beta.x * c0.x - o.beta.y * c0.y;
      r.y += o.beta.x * c0.y + o.beta.y * c0.x;
    }
    *c = r;
  }
}

// C from the FP32 partials part[z][n'][m'], one thread per output (few
// partials).  op(A) = A^H: Re = C'[2m][2n] + C'[2m+1][2n+1], Im = C'[2m][2n+1]
// - C'[2m+1][2n] (M' = 2M, N' = 2N); op(A) = A: (C'[m][2n], C'[m][2n+1]).
template <bool CONJ>
__global__ void k_x3_reduce(const float* __restrict__ part, int nz, int M, int N, X3Out o,
                            double2* __restrict__ C, int64_t ldc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)M * N) return;
  const int m = (int)(t % M), n = (int)(t / M);
  float re = 0.f, im = 0.f;
  if (CONJ) {
    const int64_t Mr = 2 * (int64_t)M, plane = Mr * 2 * (int64_t)N;
    const float* p0 = part + (size_t)(2 * n) * Mr + 2 * m;
    const float* p1 = p0 + Mr;
    for (int z = 0; z < nz; ++z) {
      const float2 a = *(const float2*)(p0 + (size_t)z * plane);  // (2m,2n), (2m+1,2n)
      const float2 b = *(const float2*)(p1 + (size_t)z * plane);  // (2m,2n+1), (2m+1,2n+1)
      re += a.x + b.y;
      im += b.x - a.y;
    }
  } else {
    const int64_t plane = (int64_t)M * 2 * N;
    const float* p0 = part + (size_t)(2 * n) * M + m;
    for (int z = 0; z < nz; ++z) {
      re += p0[(size_t)z * plane];
      im += p0[(size_t)z * plane + M];
    }
  }
  x3_store(o, re, im, C + (size_t)n * ldc + m);
}

// The same for many partials: a block of 8 warps per 32 consecutive outputs of
// one column; warp w sums partials z = w mod 8 (four loads in flight per
// lane, coalesced across the lanes), then the warps' sums are added.
template <bool CONJ>
__global__ void __launch_bounds__(256) k_x3_reduce_wide(const float* __restrict__ part, int nz,
                                                        int M, int N, X3Out o,
                                                        double2* __restrict__ C, int64_t ldc) {
  __shared__ float2 acc[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int m = blockIdx.x * 32 + lane, n = blockIdx.y;
  float re = 0.f, im = 0.f;
  if (m < M) {
    if (CONJ) {
      const int64_t Mr = 2 * (int64_t)M, plane = Mr * 2 * (int64_t)N;
      const float* p0 = part + (size_t)(2 * n) * Mr + 2 * m;
      int z = w;
      for (; z + 24 < nz; z += 32) {
        float2 a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a[u] = *(const float2*)(p0 + (size_t)(z + 8 * u) * plane);
          b[u] = *(const float2*)(p0 + (size_t)(z + 8 * u) * plane + Mr);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          re += a[u].x + b[u].y;
          im += b[u].x - a[u].y;
        }
      }
      for (; z < nz; z += 8) {
        const float2 a = *(const float2*)(p0 + (size_t)z * plane);
        const float2 b = *(const float2*)(p0 + (size_t)z * plane + Mr);
        re += a.x + b.y;
        im += b.x - a.y;
      }
    } else {
      const int64_t plane = (int64_t)M * 2 * N;
      const float* p0 = part + (size_t)(2 * n) * M + m;
      int z = w;
      for (; z + 24 < nz; z += 32) {
        float a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a[u] = p0[(size_t)(z + 8 * u) * plane];
          b[u] = p0[(size_t)(z + 8 * u) * plane + M];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          re += a[u];
          im += b[u];
        }
      }
      for (; z < nz; z += 8) {
        re += p0[(size_t)z * plane];
        im += p0[(size_t)z * plane + M];
      }
    }
  }
  acc[w][lane] = make_float2(re, im);
  __syncthreads();
  if (w != 0 || m >= M) return;
  re = 0.f;
  im = 0.f;
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    re += acc[v][lane].x;
    im += acc[v][lane].y;
  }
  x3_store(o, re, im, C + (size_t)n * ldc + m);
}

// FP32 accumulation in tensor memory rounds once per 16-wide MMA and not to
// nearest, so its error grows with the accumulated length: the leading
// product runs in partials of kX3Kps0 K blocks (512 real K), the five smaller
// ones (at most 2^-8 of it) in long partials.  Partials above kX3PartCap run as
// K segments added into C.
constexpr int kX3Kps0 = 8;
constexpr size_t kX3PartCap = (size_t)1 << 30;

struct X3Geom {
  int64_t Mr, Nr, seg, pitch, tiles;
  int kb_seg, z_rest, kps_rest, z0;
  size_t bytes_a, bytes_b, bytes_p;
};
static X3Geom x3_geom(bool conjA, int M, int N, int K) {
  X3Geom g;
  g.Mr = conjA ? 2 * (int64_t)M : M;
  g.Nr = 2 * (int64_t)N;
  const int64_t Kr = conjA ? K : 2 * (int64_t)K;
  g.seg = round_up(std::max<int64_t>(Kr, 1), TC_BK);
  g.kb_seg = (int)(g.seg / TC_BK);
  g.pitch = X3_S * g.seg;
  const int kb_rest = (X3_TERMS - 1) * g.kb_seg;
  // the long ranges spread over about two waves of output tiles, at least 8
  // blocks each; every range gets at least one block
  const int64_t tiles = ((g.Mr + TC_BM - 1) / TC_BM) * ((g.Nr + TC_BN - 1) / TC_BN);
  g.tiles = tiles;
  int nz = (int)std::max<int64_t>(1, std::min<int64_t>((2 * 152 + tiles - 1) / tiles, kb_rest / 8));
  g.kps_rest = (kb_rest + nz - 1) / nz;
  g.z_rest = (kb_rest + g.kps_rest - 1) / g.kps_rest;
  g.z0 = (g.kb_seg + kX3Kps0 - 1) / kX3Kps0;
  g.bytes_a = align256((size_t)g.Mr * g.pitch * 2);
  g.bytes_b = align256((size_t)g.Nr * g.pitch * 2);
  g.bytes_p = (size_t)(g.z_rest + g.z0) * g.Mr * g.Nr * sizeof(float);
  return g;
}

// One K segment.
static void x3_gemm_seg(System& s, bool conjA, int M, int N, int K, double2 alpha,
                        const double2* A, int64_t lda, const double2* B, int64_t ldb, double2 beta,
                        double2* C, int64_t ldc, cudaStream_t st) {
  const X3Geom g = x3_geom(conjA, M, N, K);
  const int64_t Mr = g.Mr, Nr = g.Nr, seg = g.seg, pitch = g.pitch;
  const int nz = g.z_rest + g.z0;
  ensure(s.ws_oz, g.bytes_a + g.bytes_b + g.bytes_p);
  char* base = s.ws_oz.p;
  const __nv_bfloat16* pA = (__nv_bfloat16*)base;
  __nv_bfloat16* pB = (__nv_bfloat16*)(base + g.bytes_a);
  float* part = (float*)(base + g.bytes_a + g.bytes_b);

  TimedScope ts(s, KF_GEMM_X3, st, 2.0 * X3_TERMS * (double)Mr * Nr * (double)seg,
                16.0 * (double)M * K + 16.0 * (double)K * N + 4.0 * X3_S * ((double)Mr + Nr) * seg +
                    8.0 * nz * (double)Mr * Nr + 16.0 * (double)M * N);
  {
    __nv_bfloat16* wA = (__nv_bfloat16*)s.ws_oz.p;
    if (conjA)
      k_x3_slice_cols<X3_S><<<dim3((unsigned)((seg / 2 + 255) / 256), M), 256, 0, st>>>(A, lda, K, (int)seg,
                                                                                wA, pitch);
    else
      k_x3_slice_rows<X3_S><<<dim3((M + 31) / 32, (unsigned)((seg / 2 + 31) / 32)), 256, 0, st>>>(
          A, lda, M, K, (int)seg, wA, pitch);
    PWH_LAUNCH_CHECK();
  }
  if (conjA) {
    k_x3_slice_cols<X3_S><<<dim3((unsigned)((seg / 2 + 255) / 256), N), 256, 0, st>>>(B, ldb, K, (int)seg,
                                                                              pB, pitch);
    PWH_LAUNCH_CHECK();
  } else {
    k_x3_slice_b2<X3_S><<<dim3((unsigned)((seg / 2 + 255) / 256), N), 256, 0, st>>>(B, ldb, K, (int)seg,
                                                                            pB, pitch);
    PWH_LAUNCH_CHECK();
  }
  CUtensorMap ma = make_map(pA, Mr, pitch, pitch, TC_BM);
  CUtensorMap mb = make_map(pB, Nr, pitch, pitch, TC_BN);
  TcArgs a{};
  a.M = (int)Mr;
  a.N = (int)Nr;
  a.kb_seg = g.kb_seg;
  a.terms = X3_TERMS;
  a.kb_per_split = g.kps_rest;
  a.z_rest = g.z_rest;
  a.kps0 = kX3Kps0;
  a.part = part;
  a.err = device_error_word(s);
  a.oz = 2;
  // slice pairs (s, t) with s + t <= 2, the leading pair first
  const unsigned char ta[X3_TERMS] = {0, 0, 1, 0, 1, 2}, tb[X3_TERMS] = {0, 1, 0, 2, 1, 0};
  for (int p = 0; p < X3_TERMS; ++p) {
    a.oz_a[p] = ta[p];
    a.oz_b[p] = tb[p];
  }
  dim3 grid((unsigned)((Mr + TC_BM - 1) / TC_BM), (unsigned)((Nr + TC_BN - 1) / TC_BN), nz);
  tc_launch<0>(ma, mb, a, grid, st);
  PWH_LAUNCH_CHECK();
  X3Out o;
  o.alpha = alpha;
  o.beta = beta;
  o.af = (float)alpha.x;
  const bool ar = alpha.y == 0.0 && (double)o.af == alpha.x;
  o.mode = ar && beta.x == 0.0 && beta.y == 0.0 ? 0 : ar && beta.x == 1.0 && beta.y == 0.0 ? 1 : 2;
  const int64_t tot = (int64_t)M * N;
  if (nz > 8 && N <= 65535) {
    const dim3 rg((unsigned)((M + 31) / 32), (unsigned)N);
    if (conjA)
      k_x3_reduce_wide<true><<<rg, 256, 0, st>>>(part, nz, M, N, o, C, ldc);
    else
      k_x3_reduce_wide<false><<<rg, 256, 0, st>>>(part, nz, M, N, o, C, ldc);
  } else if (conjA) {
    k_x3_reduce<true><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(part, nz, M, N, o, C, ldc);
  } else {
    k_x3_reduce<false><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(part, nz, M, N, o, C, ldc);
  }
  PWH_LAUNCH_CHECK();
}

// K per segment: whole 512-wide real ranges (512 complex K for A^H B, 256 for
// A B) while the partials of the whole product pass the cap.
static int x3_kseg(bool conjA, int M, int N, int K) {
  const X3Geom g = x3_geom(conjA, M, N, K);
  if (g.bytes_p <= kX3PartCap) return K;
  // one short partial per 512 real K, at most 2 * 152 / tiles long ones
  const size_t plane = (size_t)g.Mr * g.Nr * sizeof(float);
  const int64_t units =
      std::max<int64_t>(1, (int64_t)(kX3PartCap / plane) - (2 * 152 + g.tiles - 1) / g.tiles);
  return (int)std::min<int64_t>(K, units * (conjA ? 512 : 256));
}

void x3_reserve(System& s, bool conjA, int M, int N, int K) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  // the first segment is the largest
  const X3Geom g = x3_geom(conjA, M, N, x3_kseg(conjA, M, N, K));
  ensure(s.ws_oz, g.bytes_a + g.bytes_b + g.bytes_p);
}

// ---- 16-bit sliced complex GEMM (the reduced-precision phase's subspace
// products): each operand value rounded to FP32 and cut to its two leading
// BF16 slices [hi | lo] (about 16 significant bits, the accuracy of the
// split-BF16 projector GEMMs of the reduced-precision H), the three products
// hi.hi + hi.lo + lo.hi in one BF16 GEMM (the projector GEMM's operand
// layout), FP32 accumulation in tensor memory over K ranges of at most
// kX2Kmax real K (the tensor core's truncating accumulation stays below the
// slices' own rounding there), FP32 reduction of the partials.
constexpr int X2_S = 2, X2_TERMS = 3;
constexpr int kX2Kmax = 8192;
struct X2Geom {
  int64_t Mr, Nr, seg, pitch, tiles;
  int kb_seg, kps, nz;
  size_t bytes_a, bytes_b, bytes_p;
};
static X2Geom x2_geom(bool conjA, int M, int N, int K) {
  X2Geom g;
  g.Mr = conjA ? 2 * (int64_t)M : M;
  g.Nr = 2 * (int64_t)N;
  const int64_t Kr = conjA ? K : 2 * (int64_t)K;
  g.seg = round_up(std::max<int64_t>(Kr, 1), TC_BK);
  g.kb_seg = (int)(g.seg / TC_BK);
  g.pitch = X2_S * g.seg;
  const int kb_total = X2_TERMS * g.kb_seg;
  g.tiles = ((g.Mr + TC_BM - 1) / TC_BM) * ((g.Nr + TC_BN - 1) / TC_BN);
  // K ranges: at least enough that none exceeds kX2Kmax real K (accuracy),
  // then the count with the least modelled time (waves of CTAs, one per SM at
  // a time, times a CTA's share of its tile's K and about 2 us of set-up and
  // epilogue, plus the partials written and read once more; nominal rates
  // 2.25 PFLOP/s BF16, 7.9 TB/s)
  const int nz_acc = std::max(1, (kb_total + kX2Kmax / TC_BK - 1) / (kX2Kmax / TC_BK));
  const double tile_s = 2.0 * TC_BM * TC_BN * TC_BK * (double)kb_total / (2.25e15 / 152);
  const double part_s = 2.0 * (double)g.Mr * g.Nr * sizeof(float) / 7.9e12;
  int nz = std::min(kb_total, nz_acc);
  double best = 1e300;
  for (int z = nz_acc; z <= std::min(kb_total, std::max(nz_acc, 1024)); ++z) {
    const double waves = (double)((g.tiles * z + 151) / 152);
    const double t = waves * (tile_s / z + 2e-6) + z * part_s;
    if (t < best) {
      best = t;
      nz = z;
    }
  }
  g.kps = (kb_total + nz - 1) / nz;
  g.nz = (kb_total + g.kps - 1) / g.kps;
  g.bytes_a = align256((size_t)g.Mr * g.pitch * 2);
  g.bytes_b = align256((size_t)g.Nr * g.pitch * 2);
  g.bytes_p = (size_t)g.nz * g.Mr * g.Nr * sizeof(float);
  return g;
}

static void x2_gemm_seg(System& s, bool conjA, int M, int N, int K, double2 alpha,
                        const double2* A, int64_t lda, const double2* B, int64_t ldb, double2 beta,
                        double2* C, int64_t ldc, cudaStream_t st) {
  const X2Geom g = x2_geom(conjA, M, N, K);
  const int64_t Mr = g.Mr, Nr = g.Nr, seg = g.seg, pitch = g.pitch;
  ensure(s.ws_oz, g.bytes_a + g.bytes_b + g.bytes_p);
  char* base = s.ws_oz.p;
  __nv_bfloat16* pA = (__nv_bfloat16*)base;
  __nv_bfloat16* pB = (__nv_bfloat16*)(base + g.bytes_a);
  float* part = (float*)(base + g.bytes_a + g.bytes_b);
  TimedScope ts(s, KF_GEMM_X3, st, 2.0 * X2_TERMS * (double)Mr * Nr * (double)seg,
                16.0 * (double)M * K + 16.0 * (double)K * N + 4.0 * X2_S * ((double)Mr + Nr) * seg +
                    8.0 * g.nz * (double)Mr * Nr + 16.0 * (double)M * N);
  if (conjA) {
    k_x3_slice_cols<X2_S><<<dim3((unsigned)((seg / 2 + 255) / 256), M), 256, 0, st>>>(A, lda, K, (int)seg,
                                                                                    pA, pitch);
    PWH_LAUNCH_CHECK();
    k_x3_slice_cols<X2_S><<<dim3((unsigned)((seg / 2 + 255) / 256), N), 256, 0, st>>>(B, ldb, K, (int)seg,
                                                                                    pB, pitch);
  } else {
    k_x3_slice_rows<X2_S><<<dim3((M + 31) / 32, (unsigned)((seg / 2 + 31) / 32)), 256, 0, st>>>(
        A, lda, M, K, (int)seg, pA, pitch);
    PWH_LAUNCH_CHECK();
    k_x3_slice_b2<X2_S><<<dim3((unsigned)((seg / 2 + 255) / 256), N), 256, 0, st>>>(B, ldb, K, (int)seg,
                                                                                  pB, pitch);
  }
  PWH_LAUNCH_CHECK();
  CUtensorMap ma = make_map(pA, Mr, pitch, pitch, TC_BM);
  CUtensorMap mb = make_map(pB, Nr, pitch, pitch, TC_BN);
  TcArgs a{};
  a.M = (int)Mr;
  a.N = (int)Nr;
  a.kb_seg = g.kb_seg;
  a.terms = X2_TERMS;   // hi.hi + hi.lo + lo.hi over the [hi | lo] segments
  a.kb_per_split = g.kps;
  a.part = part;
  a.err = device_error_word(s);
  a.oz = 0;
  dim3 grid((unsigned)((Mr + TC_BM - 1) / TC_BM), (unsigned)((Nr + TC_BN - 1) / TC_BN), g.nz);
  tc_launch<0>(ma, mb, a, grid, st);
  PWH_LAUNCH_CHECK();
  X3Out o;
  o.alpha = alpha;
  o.beta = beta;
  o.af = (float)alpha.x;
  const bool ar = alpha.y == 0.0 && (double)o.af == alpha.x;
  o.mode = ar && beta.x == 0.0 && beta.y == 0.0 ? 0 : ar && beta.x == 1.0 && beta.y == 0.0 ? 1 : 2;
  const int64_t tot = (int64_t)M * N;
  if (g.nz > 8 && N <= 65535) {
    const dim3 rg((unsigned)((M + 31) / 32), (unsigned)N);
    if (conjA)
      k_x3_reduce_wide<true><<<rg, 256, 0, st>>>(part, g.nz, M, N, o, C, ldc);
    else
      k_x3_reduce_wide<false><<<rg, 256, 0, st>>>(part, g.nz, M, N, o, C, ldc);
  } else if (conjA) {
    k_x3_reduce<true><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(part, g.nz, M, N, o, C, ldc);
  } else {
    k_x3_reduce<false><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(part, g.nz, M, N, o, C, ldc);
  }
  PWH_LAUNCH_CHECK();
}

// K per segment so that the partials of one segment stay under kX3PartCap.
static int x2_kseg(bool conjA, int M, int N, int K) {
  const X2Geom g = x2_geom(conjA, M, N, K);
  if (g.bytes_p <= kX3PartCap) return K;
  const size_t plane = (size_t)g.Mr * g.Nr * sizeof(float);
  const int64_t nzmax = std::max<int64_t>(1, (int64_t)(kX3PartCap / plane));
  // real K a segment may take: nzmax ranges of kX2Kmax / 3 (three products)
  const int64_t kr = std::max<int64_t>(TC_BK, nzmax * (kX2Kmax / X2_TERMS) / TC_BK * TC_BK);
  return (int)std::max<int64_t>(1, std::min<int64_t>(K, conjA ? kr : kr / 2));
}

void x2_gemm(System& s, bool conjA, int M, int N, int K, double2 alpha, const double2* A,
             int64_t lda, const double2* B, int64_t ldb, double2 beta, double2* C, int64_t ldc,
             cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_tc_gemm<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  });
  const int kseg = x2_kseg(conjA, M, N, K);
  for (int k0 = 0; k0 == 0 || k0 < K; k0 += kseg) {
    const int kk = std::min(kseg, K - k0);
    x2_gemm_seg(s, conjA, M, N, kk, alpha, A + (conjA ? (int64_t)k0 : (int64_t)k0 * lda), lda,
                B + k0, ldb, k0 == 0 ? beta : make_double2(1, 0), C, ldc, st);
  }
}

void x3_gemm(System& s, bool conjA, int M, int N, int K, double2 alpha, const double2* A,
             int64_t lda, const double2* B, int64_t ldb, double2 beta, double2* C, int64_t ldc,
             cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_tc_gemm<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  });
  const int kseg = x3_kseg(conjA, M, N, K);
  for (int k0 = 0; k0 == 0 || k0 < K; k0 += kseg) {
    const int kk = std::min(kseg, K - k0);
    x3_gemm_seg(s, conjA, M, N, kk, alpha, A + (conjA ? (int64_t)k0 : (int64_t)k0 * lda), lda,
                B + k0, ldb, k0 == 0 ? beta : make_double2(1, 0), C, ldc, st);
  }
}

}  // namespace pwh
