// Complex GEMM on the CUDA cores (FP64 and FP32):
//     C = alpha * op(A) * B + beta * C,   op(A) = A or A^H,
// all matrices column-major complex with explicit leading dimensions.  It
// serves the projector products p_ij = <beta_j|psi_i> ("becp") and the
// back-projection of the nonlocal term (Eq. pauli_ks), and the subspace
// matrices O_ij = <psi_i|O|psi_j> and Ritz rotations of the eigensolver (Sec.
// "New parallelization levels").  There is no FP64 tensor-core path on this
// GPU; the FP64 operator is bound by the FP64 pipe.
//
// Output tiles of BM x BN per 256-thread block with TM x TN complex outputs per
// thread, shaped by the width of the product (see cgemm_impl).  A long
// reduction (K = npw) with few output tiles is split over blockIdx.z into a
// workspace and summed by k_splitk_reduce in a fixed order (deterministic).
#include <algorithm>
#include <cstdlib>

#include "common.cuh"
#include "gemm.cuh"

namespace pwh {

// TS: storage type of A, B, C and the split-K partials; T: compute type
// (operands are rounded to T when staged in shared memory, products are
// accumulated in T).  BM x BN output tile per 256-thread block, TM x TN
// complex outputs per thread (thread (tx, ty) owns rows tx + (BM/TM) i and
// columns ty + (BN/TN) j), K-slabs of BK: the next slab is fetched into
// registers while the current one is multiplied out of shared memory.
template <typename TS, typename T, bool CONJ_A, int BM, int BN, int TM, int TN, int BK>
__global__ void __launch_bounds__(256) k_cgemm(int M, int N, int K, const cx<TS>* __restrict__ A,
                                               int64_t lda, const cx<TS>* __restrict__ B,
                                               int64_t ldb, cx<TS>* __restrict__ C, int64_t ldc,
                                               cx<TS> alpha, cx<TS> beta, int kchunk,
                                               cx<TS>* __restrict__ part) {
  constexpr int NTX = BM / TM, NTY = BN / TN;
  static_assert(NTX * NTY == 256, "256 threads");
  constexpr int LA = (BM * BK + 255) / 256, LB = (BN * BK + 255) / 256;
  __shared__ cx<T> As[BK][BM + 1];
  __shared__ cx<T> Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kb = blockIdx.z * kchunk;
  const int ke = min(K, kb + kchunk);
  cx<T> acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = mk<T>(0, 0);
  cx<T> ra[LA], rb[LB];
  // slab k0 of op(A) and B into registers, rounded to T (zero outside the
  // matrices)
  auto fetch = [&](int k0) {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + 256 * r;
      cx<TS> z = mk<TS>(0, 0);
      if (e < BM * BK) {
        int m, k;
        if (!CONJ_A) { m = e % BM; k = e / BM; } else { k = e % BK; m = e / BK; }
        const int gm = m0 + m, gk = k0 + k;
        if (gm < M && gk < ke) z = CONJ_A ? A[(size_t)gm * lda + gk] : A[(size_t)gk * lda + gm];
      }
      ra[r] = mk<T>((T)z.x, CONJ_A ? -(T)z.y : (T)z.y);
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      const int e = tid + 256 * r;
      cx<TS> z = mk<TS>(0, 0);
      if (e < BN * BK) {
        const int k = e % BK, n = e / BK;
        const int gn = n0 + n, gk = k0 + k;
        if (gn < N && gk < ke) z = B[(size_t)gn * ldb + gk];
      }
      rb[r] = mk<T>((T)z.x, (T)z.y);
    }
  };
  auto stage = [&]() {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + 256 * r;
      if (e < BM * BK) {
        int m, k;
        if (!CONJ_A) { m = e % BM; k = e / BM; } else { k = e % BK; m = e / BK; }
        As[k][m] = ra[r];
      }
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      const int e = tid + 256 * r;
      if (e < BN * BK) {
        const int k = e % BK, n = e / BK;
        Bs[k][n] = rb[r];
      }
    }
  };
  if (kb < ke) fetch(kb);
  for (int k0 = kb; k0 < ke; k0 += BK) {
    stage();
    __syncthreads();
    if (k0 + BK < ke) fetch(k0 + BK);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      cx<T> a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[k][tx + NTX * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[k][ty + NTY * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          acc[i][j].x = fma(a[i].x, b[j].x, acc[i][j].x);
          acc[i][j].x = fma(-a[i].y, b[j].y, acc[i][j].x);
          acc[i][j].y = fma(a[i].x, b[j].y, acc[i][j].y);
          acc[i][j].y = fma(a[i].y, b[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gm = m0 + tx + NTX * i, gn = n0 + ty + NTY * j;
      if (gm < M && gn < N) {
        const cx<TS> v = mk<TS>((TS)acc[i][j].x, (TS)acc[i][j].y);
        if (part) {
          part[((size_t)blockIdx.z * N + gn) * M + gm] = v;
        } else {
          cx<TS> r = mul<TS>(alpha, v);
          if (beta.x != (TS)0 || beta.y != (TS)0) r = add<TS>(r, mul<TS>(beta, C[(size_t)gn * ldc + gm]));
          C[(size_t)gn * ldc + gm] = r;
        }
      }
    }
}

// C = alpha * sum_z part[z] (* rowscale[m] if given) + beta * C, summed in
// the fixed order z = 0, 1, ... (deterministic).  Grid-stride over outputs,
// four partials in flight a thread.
template <typename T>
__global__ void k_splitk_reduce(int M, int N, int nsplit, const cx<T>* __restrict__ part,
                                cx<T>* __restrict__ C, int64_t ldc, cx<T> alpha, cx<T> beta,
                                const double* __restrict__ rowscale) {
  const int64_t tot = (int64_t)M * N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    cx<T> s = mk<T>(0, 0);
    int z = 0;
    for (; z + 3 < nsplit; z += 4) {
      const cx<T> p0 = part[(size_t)z * tot + t], p1 = part[(size_t)(z + 1) * tot + t];
      const cx<T> p2 = part[(size_t)(z + 2) * tot + t], p3 = part[(size_t)(z + 3) * tot + t];
      s = add<T>(add<T>(add<T>(add<T>(s, p0), p1), p2), p3);
    }
    for (; z < nsplit; ++z) s = add<T>(s, part[(size_t)z * tot + t]);
    const int m = (int)(t % M), n = (int)(t / M);
    if (rowscale) s = scl<T>(s, (T)rowscale[m]);
    cx<T> r = mul<T>(alpha, s);
    if (beta.x != (T)0 || beta.y != (T)0) r = add<T>(r, mul<T>(beta, C[(size_t)n * ldc + m]));
    C[(size_t)n * ldc + m] = r;
  }
}

// The same for long reductions of few outputs (many partials): a block takes
// 32 consecutive outputs, its 8 warps sum z = g, g + 8, ... and the 8 group
// sums are added in a fixed order (deterministic).
template <typename T>
__global__ void __launch_bounds__(256) k_splitk_reduce_wide(int M, int N, int nsplit,
                                                            const cx<T>* __restrict__ part,
                                                            cx<T>* __restrict__ C, int64_t ldc,
                                                            cx<T> alpha, cx<T> beta,
                                                            const double* __restrict__ rowscale) {
  __shared__ cx<T> red[8][32];
  const int64_t tot = (int64_t)M * N;
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int64_t t = (int64_t)blockIdx.x * 32 + lane;
  cx<T> acc = mk<T>(0, 0);
  if (t < tot) {
    int z = g;
    for (; z + 24 < nsplit; z += 32) {
      const cx<T> p0 = part[(size_t)z * tot + t], p1 = part[(size_t)(z + 8) * tot + t];
      const cx<T> p2 = part[(size_t)(z + 16) * tot + t], p3 = part[(size_t)(z + 24) * tot + t];
      acc = add<T>(acc, add<T>(add<T>(p0, p1), add<T>(p2, p3)));
    }
    for (; z < nsplit; z += 8) acc = add<T>(acc, part[(size_t)z * tot + t]);
  }
  red[g][lane] = acc;
  __syncthreads();
  if (g == 0 && t < tot) {
    cx<T> s = red[0][lane];
#pragma unroll
    for (int h = 1; h < 8; ++h) s = add<T>(s, red[h][lane]);
    const int m = (int)(t % M), n = (int)(t / M);
    if (rowscale) s = scl<T>(s, (T)rowscale[m]);
    cx<T> r = mul<T>(alpha, s);
    if (beta.x != (T)0 || beta.y != (T)0) r = add<T>(r, mul<T>(beta, C[(size_t)n * ldc + m]));
    C[(size_t)n * ldc + m] = r;
  }
}

// Tile shapes (BM, BN, TM, TN, BK) by the width N of the product: narrow
// products (a few unconverged bands) take tall thin tiles so that no
// arithmetic is spent on padding columns; FP32 takes 8 x 8 (or 8 x 4)
// outputs per thread, FP64 4 x 4 (its pipe, not shared memory, is the limit).
template <typename TS, typename T, int BM, int BN, int TM, int TN, int BK>
static void cgemm_launch(System& s, bool conjA, int M, int N, int K, cx<TS> alpha, const cx<TS>* A,
                         int64_t lda, const cx<TS>* B, int64_t ldb, cx<TS> beta, cx<TS>* C,
                         int64_t ldc, cudaStream_t st, const double* rowscale) {
  const int gm = (M + BM - 1) / BM, gn = (N + BN - 1) / BN;
  const int tiles = gm * gn;
  // split the reduction when the output tiles alone fill less than one wave
  // (into about two blocks per SM, chunks of at least 32: small square
  // products such as the eigensolver's n x n x n ones still spread out)
  // (the partials of a split stay below 64 MB)
  int nsplit = 1;
  if (tiles < 152 && K > 2 * BK) {
    nsplit = std::min((2 * 152 + tiles - 1) / tiles, std::max(1, K / 32));
    const int64_t cap = std::max<int64_t>(1, ((int64_t)64 << 20) / ((int64_t)M * N * (int64_t)sizeof(cx<TS>)));
    nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(nsplit, cap));
  }
  int kchunk = (K + nsplit - 1) / nsplit;
  kchunk = ((kchunk + BK - 1) / BK) * BK;
  nsplit = std::max(1, (K + kchunk - 1) / kchunk);
  if (K <= 0) {
    nsplit = 1;
    kchunk = 0;
  }
  const bool use_part = nsplit > 1 || rowscale != nullptr;
  cx<TS>* part = nullptr;
  if (use_part) {
    ensure(s.ws_split, (size_t)nsplit * M * N * sizeof(cx<TS>));
    part = (cx<TS>*)s.ws_split.p;
  }
  dim3 grid(gm, gn, nsplit);
  TimedScope ts(s, sizeof(T) == 8 ? KF_GEMM_FP64 : KF_GEMM_FP32, st, 8.0 * M * N * (double)K,
                sizeof(cx<TS>) * ((double)M * K + (double)K * N + 2.0 * M * N));
  if (conjA)
    k_cgemm<TS, T, true, BM, BN, TM, TN, BK><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc,
                                                                   alpha, beta, kchunk, part);
  else
    k_cgemm<TS, T, false, BM, BN, TM, TN, BK><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc,
                                                                    alpha, beta, kchunk, part);
  PWH_LAUNCH_CHECK();
  if (use_part) {
    const int64_t tot = (int64_t)M * N;
    if (nsplit >= 16 && tot <= 152 * 256) {
      k_splitk_reduce_wide<TS><<<(unsigned)((tot + 31) / 32), 256, 0, st>>>(M, N, nsplit, part, C, ldc,
                                                                           alpha, beta, rowscale);
    } else {
      const int blocks = (int)std::min<int64_t>(4 * 152, (tot + 255) / 256);
      k_splitk_reduce<TS><<<blocks, 256, 0, st>>>(M, N, nsplit, part, C, ldc, alpha, beta, rowscale);
    }
    PWH_LAUNCH_CHECK();
  }
}

template <typename TS, typename T>
static void cgemm_impl(System& s, bool conjA, int M, int N, int K, cx<TS> alpha, const cx<TS>* A,
                       int64_t lda, const cx<TS>* B, int64_t ldb, cx<TS> beta, cx<TS>* C,
                       int64_t ldc, cudaStream_t st, const double* rowscale) {
  if (M <= 0 || N <= 0) return;
  if constexpr (sizeof(T) == 4) {
    if (N > 64)
      cgemm_launch<TS, T, 128, 128, 8, 8, 16>(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, rowscale);
    else if (N > 32)
      cgemm_launch<TS, T, 128, 64, 8, 4, 8>(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, rowscale);
    else if (N > 16 && M <= 128)
      cgemm_launch<TS, T, 128, 32, 4, 4, 8>(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, rowscale);
    else if (N > 16)
      cgemm_launch<TS, T, 256, 32, 8, 4, 8>(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, rowscale);
    else if (M <= 128)
      cgemm_launch<TS, T, 128, 16, 4, 2, 8>(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, rowscale);
    else
      cgemm_launch<TS, T, 256, 16, 8, 2, 8>(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, rowscale);
  } else {
    if (N > 32)
      cgemm_launch<TS, T, 64, 64, 4, 4, 16>(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, rowscale);
    else if (N > 16)
      cgemm_launch<TS, T, 128, 32, 4, 4, 16>(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, rowscale);
    else if (N > 8)
      cgemm_launch<TS, T, 256, 16, 4, 4, 8>(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, rowscale);
    else
      cgemm_launch<TS, T, 256, 8, 4, 2, 8>(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, rowscale);
  }
}

// FP64 products of at least kOzMinFlops go to the tensor cores as sliced
// integer products (oz_gemm).

// The sliced tensor-core paths launch one block row per column of A (A^H B)
// and of B along grid y, and K / 64 blocks along grid y of the A B slicing:
// sizes past those grid limits stay on the SIMT kernels.
static bool slice_grid_ok(bool conjA, int M, int N, int K) {
  return N <= 65535 && (conjA ? M <= 65535 : K <= 65535 * 32);
}

// Whether a product of FP32-level accuracy takes the tensor-core path: large
// enough, and not too narrow.  Narrow products of moderate length stay on the
// FP32 pipe (the tensor-core path's slicing and reduction cost more than they
// save below about 48 columns of A^H B and 96 of A B at 34k plane waves).  On
// long products (K or M of at least 65,536) the tensor-core path costs about
// the slicing of the long operand whatever the width, while the FP32-pipe
// kernel reaches only about 1 TB/s: at 161,235 plane waves a 544 x 19 A^H B
// took 0.93 ms against 1.82 ms and a 161,235 x 19 x 544 A B 0.97 against
// 1.18 ms (the FP32 pipe still won at 6 columns of A B, 0.64 against 1.50).
static bool tc_width_ok(bool conjA, int M, int N, int K) {
  const int narrow = conjA ? std::min(M, N) : N;
  if (conjA ? K >= 65536 : M >= 65536) return narrow >= (conjA ? 1 : 16);
  return narrow >= (conjA ? 48 : 96);
}

template <typename T>
void cgemm(System& s, bool conjA, int M, int N, int K, cx<T> alpha, const cx<T>* A, int64_t lda,
           const cx<T>* B, int64_t ldb, cx<T> beta, cx<T>* C, int64_t ldc, cudaStream_t st,
           const double* rowscale) {
  if constexpr (sizeof(T) == 8) {
    if (K > 0 && 8.0 * M * (double)N * K >= kOzMinFlops &&
        slice_grid_ok(conjA, M, N, K)) {
      oz_gemm(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, rowscale);
      return;
    }
  }
  cgemm_impl<T, T>(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, rowscale);
}

void cgemm_f32_simt(System& s, bool conjA, int M, int N, int K, double2 alpha, const double2* A,
                    int64_t lda, const double2* B, int64_t ldb, double2 beta, double2* C,
                    int64_t ldc, cudaStream_t st) {
  cgemm_impl<double, float>(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, nullptr);
}

void cgemm_r16(System& s, bool conjA, int M, int N, int K, double2 alpha, const double2* A,
               int64_t lda, const double2* B, int64_t ldb, double2 beta, double2* C, int64_t ldc,
               cudaStream_t st) {
  // the tensor-core path above the same size and width thresholds as
  // cgemm_f32 (narrower products: the FP32 pipe, more accurate anyway)
  if (K > 0 && 8.0 * M * (double)N * K >= kX3MinFlops && tc_width_ok(conjA, M, N, K) &&
      slice_grid_ok(conjA, M, N, K)) {
    x2_gemm(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
    return;
  }
  cgemm_impl<double, float>(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, nullptr);
}

void cgemm_f32(System& s, bool conjA, int M, int N, int K, double2 alpha, const double2* A,
               int64_t lda, const double2* B, int64_t ldb, double2 beta, double2* C, int64_t ldc,
               cudaStream_t st) {
  // large products run on the tensor cores as three-slice BF16 products
  if (K > 0 && 8.0 * M * (double)N * K >= kX3MinFlops && tc_width_ok(conjA, M, N, K) &&
      slice_grid_ok(conjA, M, N, K)) {
    x3_gemm(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
    return;
  }
  cgemm_impl<double, float>(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, nullptr);
}

template void cgemm<double>(System&, bool, int, int, int, double2, const double2*, int64_t,
                            const double2*, int64_t, double2, double2*, int64_t, cudaStream_t,
                            const double*);
template void cgemm<float>(System&, bool, int, int, int, float2, const float2*, int64_t,
                           const float2*, int64_t, float2, float2*, int64_t, cudaStream_t,
                           const double*);

}  // namespace pwh

extern "C" pwh_status pwh_subspace_gemm(pwh_system* sys, int32_t precision, int32_t conj_a,
                                        int32_t M, int32_t N, int32_t K, const double* alpha,
                                        const void* A, int64_t lda, const void* B, int64_t ldb,
                                        const double* beta, void* C, int64_t ldc) {
  using namespace pwh;
  return guarded([&] {
    PWH_CHECK_ARG(sys && alpha && beta, "null argument");
    PWH_CHECK_ARG(M >= 0 && N >= 0 && K >= 0, "negative size");
    PWH_CHECK_ARG(precision == PWH_FP64 || precision == PWH_MIXED, "precision must be FP64 or MIXED");
    if (M == 0 || N == 0) return;
    PWH_CHECK_ARG(C && (K == 0 || (A && B)), "null matrix");
    PWH_CHECK_ARG(lda >= (conj_a ? K : M) && lda >= 1, "lda too small");
    PWH_CHECK_ARG(ldb >= K && ldb >= 1 && ldc >= M, "ldb or ldc too small");
    System& s = sys->s;
    const double2 al = make_double2(alpha[0], alpha[1]), be = make_double2(beta[0], beta[1]);
    if (precision == PWH_FP64)
      cgemm<double>(s, conj_a != 0, M, N, K, al, (const double2*)A, lda, (const double2*)B, ldb, be,
                    (double2*)C, ldc, s.stream);
    else
      cgemm_f32(s, conj_a != 0, M, N, K, al, (const double2*)A, lda, (const double2*)B, ldb, be,
                (double2*)C, ldc, s.stream);
  });
}
