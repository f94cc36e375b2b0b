// Small dense FP64 kernels of the Davidson subspace (dense.cu).
#pragma once
#include "common.cuh"

namespace pwh {

struct DenseWs {
  DevBuf<char> jac, chol;
  DevBuf<char> jlog;    // rotation log of the cluster and position-order Jacobi
  DevBuf<char> pj;      // position-order Jacobi: two FP32 matrices, reduction words
  DevBuf<char> ns;      // Newton-Schulz inverse square root: four k x k matrices
  double* h_word = nullptr;  // pinned host word for small device results
  void* ctl = nullptr;  // barrier words and flags of the Jacobi launch
  ~DenseWs() {
    if (jac.p) cudaFree(jac.p);
    if (chol.p) cudaFree(chol.p);
    if (jlog.p) cudaFree(jlog.p);
    if (pj.p) cudaFree(pj.p);
    if (ns.p) cudaFree(ns.p);
    if (h_word) cudaFreeHost(h_word);
    if (ctl) cudaFree(ctl);
  }
};

constexpr int kJacobiMaxN = 4096;

// Work of one sweep of the whole-GPU FP32 block Jacobi (subspaces above 512),
// in real flops.
double jacobi32_blk_sweep_flops(int n);

// Lowest nk eigenpairs of the n x n Hermitian H (ld = ldh, read only):
// theta[0..nk) ascending (device), C (n x nk, ld = n, device).  Qkeep
// (optional, ld = ldk) receives all n eigenvectors sorted by eigenvalue; with
// warm_m0 > 0 it must hold the previous call's eigenvectors of the leading
// warm_m0 x warm_m0 block of H, and the iteration starts in that basis.
// polish: FP64 result (FP32 Jacobi, then the FP64 unitary basis, Q^H H Q and
// FP64 sweeps); otherwise the FP32 result (eigenvalues to about FP32 rounding
// of ||H||, eigenvectors orthonormal to about FP32 rounding).  tol32: the
// FP32 sweeps stop at max|A_ij| <= tol32 max|A_ii| (4e-7, about five FP32
// roundings, lets one FP64 sweep finish the polish); the FP64 sweeps at
// max|A_ij| <= tol64 max|A_ii|.
void jacobi_eigh(System& s, DenseWs& w, const double2* H, int64_t ldh, int n, int nk,
                 double* theta, double2* C, cudaStream_t st, double2* Qkeep = nullptr,
                 int64_t ldk = 0, int warm_m0 = 0, bool polish = true, double tol32 = 4e-7,
                 double tol64 = 1e-13);

// FP32 stage of jacobi_eigh in one 16-CTA thread-block cluster with the matrix
// in distributed shared memory (jacobi_dsm.cu): sweeps of the n x n Hermitian
// A (FP64, ld lda) until max|A_ij| <= tol max|A_ii|; Q (ld ldq) receives the
// eigenvectors (FP64), diag the final diagonal, info[1] the sweeps, info[2]
// the rounds; the rotations of every round go to a log in w (grown here once,
// reserved by jacobi_reserve) from which a second kernel forms Q.  Returns
// false, launching nothing, when n is outside its range or the cluster cannot
// be resident.
bool jacobi32_cluster(System& s, DenseWs& w, const double2* A, int64_t lda, int n, double tol,
                      int max_sweeps, double2* Q, int64_t ldq, double* diag, int* info,
                      cudaStream_t st);
// Bytes of the rotation log of jacobi32_cluster for an n x n matrix.
size_t jacobi32_log_bytes(int n, int max_sweeps);

// Device words holding the number of FP64 / FP32 sweeps of the last jacobi_eigh.
inline int* jacobi_sweeps_word(DenseWs& w) { return (int*)w.ctl + 9; }
inline int* jacobi32_sweeps_word(DenseWs& w) { return (int*)w.ctl + 5; }

// Grow the workspaces for subspaces up to nmax and Cholesky blocks up to kmax
// (so that no allocation, hence no device-wide synchronisation, happens later).
void jacobi_reserve(DenseWs& w, int nmax, int kmax);

// Complete columns [m0, m) of a Hermitian matrix computed as V^H HV[:, m0:m].
void hermitize(double2* H, int64_t ld, int m0, int m, cudaStream_t st);

// Tr (k x k) such that T Tr has orthonormal first *kk columns (device int),
// from the Gram matrix S = T^H T; t0 (optional) = column norms before the
// projection that produced T, for the relative drop test.  fp32: Cholesky in
// FP32 arithmetic (for a Gram matrix that is itself FP32-accurate), else FP64.
void cholqr_factor(System& s, DenseWs& w, const double2* S, int k, const double* t0,
                   double drop_rel, double2* Tr, int* kk, cudaStream_t st, bool fp32 = false);

// Z = S^{-1/2} (k x k, ld k) of a Hermitian S (leading k x k block, ld lds)
// close to the identity, by the coupled Newton-Schulz iteration Y_0 = S,
// Z_0 = I, M = (3I - Z Y)/2, Y <- Y M, Z <- M Z, in FP64 (fp64) or FP32
// arithmetic.  Returns false, leaving Z untouched, unless ||S - I||_F <= 1e-2
// (then two or three steps reach the arithmetic's rounding).  Synchronises
// the stream once (to read ||S - I||_F).
bool ns_inv_sqrt(System& s, DenseWs& w, const double2* S, int64_t lds, int k, bool fp64,
                 double2* Z, cudaStream_t st);

}  // namespace pwh
