// Complex GEMM on the CUDA cores (FP64 and FP32):
//     C = alpha * op(A) * B + beta * C,   op(A) = A or A^H,
// all matrices column-major complex with explicit leading dimensions.  It
// serves the projector products p_ij = <beta_j|psi_i> ("becp") and the
// back-projection of the nonlocal term (Eq. pauli_ks), and the subspace
// matrices O_ij = <psi_i|O|psi_j> and Ritz rotations of the eigensolver (Sec.
// "New parallelization levels").  There is no FP64 tensor-core path on this
// GPU; the FP64 operator is bound by the FP64 pipe.
//
// 64x64 output tile per 256-thread block, 4x4 complex outputs per thread,
// K-slabs of 16 staged in shared memory.  A long reduction (K = npw) with few
// output tiles is split over blockIdx.z into a workspace and summed by
// k_splitk_reduce in a fixed order (deterministic).
#include <algorithm>

#include "common.cuh"
#include "gemm.cuh"

namespace pwh {

constexpr int GBM = 64, GBN = 64, GBK = 16;

// TS: storage type of A, B, C and the split-K partials; T: compute type
// (operands are rounded to T when staged in shared memory, products are
// accumulated in T).
template <typename TS, typename T, bool CONJ_A>
__global__ void __launch_bounds__(256) k_cgemm(int M, int N, int K, const cx<TS>* __restrict__ A,
                                               int64_t lda, const cx<TS>* __restrict__ B,
                                               int64_t ldb, cx<TS>* __restrict__ C, int64_t ldc,
                                               cx<TS> alpha, cx<TS> beta, int kchunk,
                                               cx<TS>* __restrict__ part) {
  __shared__ cx<T> As[GBK][GBM + 1];
  __shared__ cx<T> Bs[GBK][GBN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.x * GBM, n0 = blockIdx.y * GBN;
  const int kb = blockIdx.z * kchunk;
  const int ke = min(K, kb + kchunk);
  cx<T> acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mk<T>(0, 0);

  for (int k0 = kb; k0 < ke; k0 += GBK) {
    // A tile: op(A)[m][k] for m in [m0, m0+64), k in [k0, k0+16)
    for (int t = threadIdx.x; t < GBM * GBK; t += 256) {
      cx<T> v = mk<T>(0, 0);
      if (!CONJ_A) {
        int m = t % GBM, k = t / GBM;
        int gm = m0 + m, gk = k0 + k;
        if (gm < M && gk < ke) {
          cx<TS> z = A[(size_t)gk * lda + gm];
          v = mk<T>((T)z.x, (T)z.y);
        }
        As[k][m] = v;
      } else {
        int k = t % GBK, m = t / GBK;
        int gm = m0 + m, gk = k0 + k;
        if (gm < M && gk < ke) {
          cx<TS> z = A[(size_t)gm * lda + gk];
          v = mk<T>((T)z.x, -(T)z.y);
        }
        As[k][m] = v;
      }
    }
    for (int t = threadIdx.x; t < GBN * GBK; t += 256) {
      int k = t % GBK, n = t / GBK;
      int gn = n0 + n, gk = k0 + k;
      cx<T> v = mk<T>(0, 0);
      if (gn < N && gk < ke) {
        cx<TS> z = B[(size_t)gn * ldb + gk];
        v = mk<T>((T)z.x, (T)z.y);
      }
      Bs[k][n] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GBK; ++k) {
      cx<T> a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fma(a[i].x, b[j].x, acc[i][j].x);
          acc[i][j].x = fma(-a[i].y, b[j].y, acc[i][j].x);
          acc[i][j].y = fma(a[i].x, b[j].y, acc[i][j].y);
          acc[i][j].y = fma(a[i].y, b[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gm = m0 + tx + 16 * i, gn = n0 + ty + 16 * j;
      if (gm < M && gn < N) {
        const cx<TS> a = mk<TS>((TS)acc[i][j].x, (TS)acc[i][j].y);
        if (part) {
          part[((size_t)blockIdx.z * N + gn) * M + gm] = a;
        } else {
          cx<TS> r = mul<TS>(alpha, a);
          if (beta.x != (TS)0 || beta.y != (TS)0) r = add<TS>(r, mul<TS>(beta, C[(size_t)gn * ldc + gm]));
          C[(size_t)gn * ldc + gm] = r;
        }
      }
    }
}

// C = alpha * sum_z part[z] (* rowscale[m] if given) + beta * C
template <typename T>
__global__ void k_splitk_reduce(int M, int N, int nsplit, const cx<T>* __restrict__ part,
                                cx<T>* __restrict__ C, int64_t ldc, cx<T> alpha, cx<T> beta,
                                const double* __restrict__ rowscale) {
  int64_t tot = (int64_t)M * N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    int m = (int)(t % M), n = (int)(t / M);
    cx<T> s = mk<T>(0, 0);
    for (int z = 0; z < nsplit; ++z) s = add<T>(s, part[(size_t)z * tot + t]);
    if (rowscale) s = scl<T>(s, (T)rowscale[m]);
    cx<T> r = mul<T>(alpha, s);
    if (beta.x != (T)0 || beta.y != (T)0) r = add<T>(r, mul<T>(beta, C[(size_t)n * ldc + m]));
    C[(size_t)n * ldc + m] = r;
  }
}

template <typename TS, typename T>
static void cgemm_impl(System& s, bool conjA, int M, int N, int K, cx<TS> alpha, const cx<TS>* A,
                       int64_t lda, const cx<TS>* B, int64_t ldb, cx<TS> beta, cx<TS>* C,
                       int64_t ldc, cudaStream_t st, const double* rowscale) {
  if (M <= 0 || N <= 0) return;
  const int gm = (M + GBM - 1) / GBM, gn = (N + GBN - 1) / GBN;
  const int tiles = gm * gn;
  // split the reduction when the output alone cannot fill the GPU
  // (chunks of at least 32: small square products such as the eigensolver's
  // n x n x n ones still spread over the GPU)
  int nsplit = 1;
  if (tiles < 2 * 152 && K > 2 * GBK) {
    nsplit = std::min((2 * 152 + tiles - 1) / tiles, std::max(1, K / 32));
    nsplit = std::max(1, std::min(nsplit, 64));
  }
  int kchunk = (K + nsplit - 1) / nsplit;
  kchunk = ((kchunk + GBK - 1) / GBK) * GBK;
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
    k_cgemm<TS, T, true><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, kchunk,
                                                part);
  else
    k_cgemm<TS, T, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta,
                                                 kchunk, part);
  PWH_LAUNCH_CHECK();
  if (use_part) {
    int64_t tot = (int64_t)M * N;
    int blocks = (int)std::min<int64_t>(4096, (tot + 255) / 256);
    k_splitk_reduce<TS><<<blocks, 256, 0, st>>>(M, N, nsplit, part, C, ldc, alpha, beta, rowscale);
    PWH_LAUNCH_CHECK();
  }
}

template <typename T>
void cgemm(System& s, bool conjA, int M, int N, int K, cx<T> alpha, const cx<T>* A, int64_t lda,
           const cx<T>* B, int64_t ldb, cx<T> beta, cx<T>* C, int64_t ldc, cudaStream_t st,
           const double* rowscale) {
  cgemm_impl<T, T>(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, rowscale);
}

void cgemm_f32(System& s, bool conjA, int M, int N, int K, double2 alpha, const double2* A,
               int64_t lda, const double2* B, int64_t ldb, double2 beta, double2* C, int64_t ldc,
               cudaStream_t st) {
  cgemm_impl<double, float>(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, nullptr);
}

template void cgemm<double>(System&, bool, int, int, int, double2, const double2*, int64_t,
                            const double2*, int64_t, double2, double2*, int64_t, cudaStream_t,
                            const double*);
template void cgemm<float>(System&, bool, int, int, int, float2, const float2*, int64_t,
                           const float2*, int64_t, float2, float2*, int64_t, cudaStream_t,
                           const double*);

}  // namespace pwh
