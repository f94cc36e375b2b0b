// Internal GEMM launchers of libpwh.
#pragma once
#include "common.cuh"

namespace pwh {

// C = alpha * op(A) * B + beta * C (column-major complex); op(A) = A^H when
// conjA.  rowscale (device, length M, optional) multiplies row m of op(A)*B
// before alpha: the diagonal D of the nonlocal term.
template <typename T>
void cgemm(System& s, bool conjA, int M, int N, int K, cx<T> alpha, const cx<T>* A, int64_t lda,
           const cx<T>* B, int64_t ldb, cx<T> beta, cx<T>* C, int64_t ldc, cudaStream_t st,
           const double* rowscale = nullptr);

// Same with FP64 (complex128) storage and FP32 arithmetic: operands rounded to
// FP32, FP32 accumulation, result widened to FP64.  Products of at least
// kX3MinFlops run as x3_gemm on the tensor cores, the others on the FP32 pipe.
void cgemm_f32(System& s, bool conjA, int M, int N, int K, double2 alpha, const double2* A,
               int64_t lda, const double2* B, int64_t ldb, double2 beta, double2* C, int64_t ldc,
               cudaStream_t st);

// The same on the FP32 pipe only (round-to-nearest FP32 accumulation): for
// the small dense products of the subspace eigensolver, whose Newton-Schulz
// steps need that accuracy at K = n.
void cgemm_f32_simt(System& s, bool conjA, int M, int N, int K, double2 alpha, const double2* A,
                    int64_t lda, const double2* B, int64_t ldb, double2 beta, double2* C,
                    int64_t ldc, cudaStream_t st);

// Grow the sliced-product workspace for op(A) B of these sizes now (so that
// later products of at most this size allocate nothing).
void oz_reserve(System& s, bool conjA, int M, int N, int K);
// Products of at least this many flops (8 M N K) take oz_gemm in cgemm<double>.
constexpr double kOzMinFlops = 2e8;

// FP64-equivalent complex GEMM on the BF16 tensor cores (gemm_tc.cu): same
// contract as cgemm<double>, results within FP64-level rounding (integer
// slices of the operands, exact partial sums).
void oz_gemm(System& s, bool conjA, int M, int N, int K, double2 alpha, const double2* A,
             int64_t lda, const double2* B, int64_t ldb, double2 beta, double2* C, int64_t ldc,
             cudaStream_t st, const double* rowscale = nullptr);

// FP32-equivalent complex GEMM on the BF16 tensor cores (gemm_tc.cu): same
// contract as cgemm_f32 (operands rounded to FP32), each operand value as
// three BF16 slices, six slice products accumulated in FP32.
void x3_gemm(System& s, bool conjA, int M, int N, int K, double2 alpha, const double2* A,
             int64_t lda, const double2* B, int64_t ldb, double2 beta, double2* C, int64_t ldc,
             cudaStream_t st);
// Grow the workspace x3_gemm shares with oz_gemm for op(A) B of these sizes.
void x3_reserve(System& s, bool conjA, int M, int N, int K);
// 16-bit complex GEMM on the tensor cores (two BF16 slices per FP32-rounded
// value, three slice products, about 1.5e-5 relative accuracy): the
// reduced-precision phase's subspace products, whose operator is itself
// accurate to the split-BF16 projector GEMMs.
void x2_gemm(System& s, bool conjA, int M, int N, int K, double2 alpha, const double2* A,
             int64_t lda, const double2* B, int64_t ldb, double2 beta, double2* C, int64_t ldc,
             cudaStream_t st);
// x2_gemm above the cgemm_f32 thresholds, the FP32 SIMT GEMM below them.
void cgemm_r16(System& s, bool conjA, int M, int N, int K, double2 alpha, const double2* A,
               int64_t lda, const double2* B, int64_t ldb, double2 beta, double2* C, int64_t ldc,
               cudaStream_t st);
// Products of at least this many flops (8 M N K) take x3_gemm in cgemm_f32.
constexpr double kX3MinFlops = 4e8;

}  // namespace pwh
