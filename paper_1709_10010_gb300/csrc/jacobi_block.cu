// FP32 block Jacobi for the subspace diagonalisation of the block Davidson
// method (Sec. "New parallelization levels": the O_ij = <psi_i|O|psi_j>
// matrices and their diagonalization), in one 16-CTA thread-block cluster
// with the matrix in distributed shared memory.
//
// The indices 0..N-1 (N = 32 b, the matrix zero-padded from n) form 32 blocks
// of b consecutive indices.  A round-robin tournament pairs the blocks: 31
// rounds a sweep, 16 disjoint block pairs a round, CTA c working on pair c
// (tournament positions c and 31 - c).  In a round every CTA
//   * takes the 2b x 2b diagonal block S of its pair from the columns it holds
//     and runs one cyclic Jacobi sweep over S (2b - 1 inner rounds inside the
//     CTA), accumulating the unitary V with V^H S V nearly diagonal, then one
//     Newton-Schulz step on V;
//   * publishes V; after a cluster barrier it applies A <- J^H A J, J the
//     direct sum of every pair's V, to its own 2b columns: X <- X V_c, then
//     for each pair d the rows of d's blocks, X[L_d] <- V_d^H X[L_d];
//   * sends its two blocks of columns to the CTAs of their next tournament
//     positions (every position but 0 steps forward, 31 wraps to 1); a second
//     cluster barrier ends the round.
// One inner sweep per block pair converges in as many outer sweeps as the
// scalar cyclic Jacobi needs sweeps, with 31 cluster rounds a sweep instead
// of n - 1.  Every V goes to a log; k_bjacobi_qlog forms Q = J_0 J_1 ...
// afterwards over the whole GPU.  Padded indices (n <= g < N) have zero rows
// and columns, so their rotations are exact identities and they never mix.
//
// Block buffers, published V's and the convergence words alternate between
// two copies by round parity.  No software spin: only the hardware cluster
// barrier, with control flow that every CTA derives from the same published
// numbers.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "common.cuh"
#include "dense.cuh"
#include "jacobi_rot.cuh"

namespace cg = cooperative_groups;

namespace pwh {

constexpr int kBjCluster = 16;
constexpr int kBjThreads = 768;  // 2N items of the column update, N <= 384
constexpr int kBjMaxB = 12;              // n <= 384
constexpr int kBjMaxTb = 2 * kBjMaxB;
constexpr int kBjStage = 4;              // remote V's staged at a time

struct BjArgs {
  const double2* A;  // n x n Hermitian start (full), ld lda
  int64_t lda;
  double* diag;      // out: final diagonal, n
  int* info;         // out: [0] = 0, [1] = sweeps, [2] = rounds logged
  float2* logV;      // out: V of round t, pair d at [(t 16 + d) (2b)^2], row-major
  int* logB;         // out: blocks of round t, pair d at [t 16 + d]: b0 | b1 << 16
  int64_t log_rounds;
  int n, b, max_sweeps;
  float tol;
};

// shared memory, in this order (float2 unless noted):
//   blk [2 parity][2 slots][b][N]      columns of the CTA's two blocks
//   S   [2b][2b + 1]                   the pair's diagonal block
//   V   [2b][2b]                       its accumulated rotation
//   Vp  [2 parity][2b][2b]             V published for the other CTAs
//   Vst [kBjStage][2b][2b]             remote V's staged for the row update
//   rin [b] float4                     the inner round's rotations
//   red [2 parity][2] + [64] float     convergence words and partials
__host__ __device__ inline size_t bj_smem_bytes(int b) {
  const size_t N = 32 * (size_t)b, tb = 2 * (size_t)b;
  return (4 * b * N + tb * (tb + 1) + tb * tb * (3 + kBjStage)) * 8 + (size_t)b * 16 +
         (4 + 64) * 4;
}

__device__ __forceinline__ int bj_pair(int x) { return x < 16 ? x : 31 - x; }
__device__ __forceinline__ int bj_next(int x) { return x == 0 ? 0 : (x == 31 ? 1 : x + 1); }
// index standing at position x in round r of a sweep over np players
__device__ __forceinline__ int bj_player(int x, int r, int np) {
  return x == 0 ? 0 : 1 + (x - 1 - r + (np - 1)) % (np - 1);
}

__global__ void __launch_bounds__(kBjThreads, 1) k_bjacobi_dsm(BjArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char bsm[];
  const int n = a.n, b = a.b, N = 32 * b, tb = 2 * b, tb2 = tb * tb, ldS = tb + 1;
  const int me = (int)cluster.block_rank();
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
  float2* blk = (float2*)bsm;
  float2* S = blk + (size_t)4 * b * N;
  float2* V = S + (size_t)tb * ldS;
  float2* Vp = V + tb2;
  float2* Vst = Vp + 2 * tb2;
  float4* rin = (float4*)(Vst + (size_t)kBjStage * tb2);
  float* red = (float*)(rin + b);
  const size_t slotsz = (size_t)b * N;                   // one block of columns
  const int pos0 = me, pos1 = 31 - me;                   // own positions (slots 0, 1)
  const float2 z = make_float2(0.f, 0.f);

  // ---- load: position x holds block x at round 0
  for (size_t e = tid; e < 2 * slotsz; e += nth) {
    const int s = (int)(e / slotsz);
    const size_t w = e - s * slotsz;
    const int j = (int)(w / N), i = (int)(w - (size_t)j * N);
    const int g = (s == 0 ? pos0 : pos1) * b + j;
    float2 v = z;
    if (g < n && i < n) {
      const double2 d = a.A[(size_t)g * a.lda + i];
      v = make_float2((float)d.x, (float)d.y);
    }
    blk[e] = v;
  }
  __syncthreads();

  int sweep = 0, t = 0;
  float goff = 0.f, gdm = 0.f;
  while (true) {
    for (int r = 0; r < 31; ++r, ++t) {
      const int par = t & 1;
      float2* cur = blk + (size_t)par * 2 * slotsz;
      const int P0 = bj_player(pos0, r, 32), P1 = bj_player(pos1, r, 32);
      // local index u of the pair: u < b -> block P0, else block P1; the
      // column of u is column u % b of slot u / b
      auto gl = [&](int u) { return u < b ? P0 * b + u : P1 * b + (u - b); };
      auto col = [&](int u) { return cur + (size_t)u * N; };  // slots are consecutive

      // (1) S = A[L, L] and V = I
      for (int e = tid; e < tb2; e += nth) {
        const int u = e % tb, v = e / tb;
        S[u * ldS + v] = col(v)[gl(u)];
        V[e] = make_float2(u == v ? 1.f : 0.f, 0.f);  // V[row u'][col v'] at u' tb + v'
      }
      __syncthreads();
      // (2) one cyclic sweep over S: 2b - 1 inner rounds of b disjoint pairs
      for (int ri = 0; ri < tb - 1; ++ri) {
        if (tid < b) {
          int p = bj_player(tid, ri, tb), q = bj_player(tb - 1 - tid, ri, tb);
          if (p > q) {
            const int x = p; p = q; q = x;
          }
          float c;
          float2 sv;
          jacobi_rotation_fast(S[p * ldS + q], S[p * ldS + p].x, S[q * ldS + q].x, c, sv);
          rin[tid] = make_float4(sv.x, sv.y, c, __int_as_float(p | (q << 16)));
        }
        __syncthreads();
        // S <- J^H S J on 2 x 2 blocks (row pair k, column pair l)
        for (int e = tid; e < b * b; e += nth) {
          const int k = e % b, l = e / b;
          const float4 Rk = rin[k], Rl = rin[l];
          const int pqk = __float_as_int(Rk.w), pql = __float_as_int(Rl.w);
          const int pk = pqk & 0xffff, qk = pqk >> 16, pl = pql & 0xffff, ql = pql >> 16;
          float2 y00, y01, y10, y11;
          jacobi_block<float>(S[pk * ldS + pl], S[pk * ldS + ql], S[qk * ldS + pl],
                              S[qk * ldS + ql], Rk.z, make_float2(Rk.x, Rk.y), Rl.z,
                              make_float2(Rl.x, Rl.y), y00, y01, y10, y11);
          if (k == l) {
            // the rotated pair: real diagonal, its element zeroed
            y00.y = 0.f;
            y11.y = 0.f;
            y01 = z;
            y10 = z;
          }
          S[pk * ldS + pl] = y00;
          S[pk * ldS + ql] = y01;
          S[qk * ldS + pl] = y10;
          S[qk * ldS + ql] = y11;
        }
        // V <- V J: row u, pair l
        for (int e = tid; e < tb * b; e += nth) {
          const int u = e % tb, l = e / tb;
          const float4 Rl = rin[l];
          const int pql = __float_as_int(Rl.w);
          const int pl = pql & 0xffff, ql = pql >> 16;
          const float2 sl = make_float2(Rl.x, Rl.y);
          const float2 v0 = V[u * tb + pl], v1 = V[u * tb + ql];
          V[u * tb + pl] = add<float>(scl<float>(v0, Rl.z), mul<float>(v1, make_float2(-sl.x, sl.y)));
          V[u * tb + ql] = add<float>(mul<float>(v0, sl), scl<float>(v1, Rl.z));
        }
        __syncthreads();
      }
      // (3) one Newton-Schulz step towards the nearest unitary, V (3I - V^H V)/2
      //     (the product of 2b - 1 FP32 rotation steps drifts from unitary by
      //     more than one rotation; a congruence by a non-unitary V would move
      //     the eigenvalues), published (and logged) for the other CTAs; S,
      //     free after the inner sweep, holds (3I - V^H V)/2
      for (int e = tid; e < tb2; e += nth) {
        const int u = e % tb, v = e / tb;
        float2 g = z;
        for (int k = 0; k < tb; ++k) g = add<float>(g, mulc<float>(V[k * tb + v], V[k * tb + u]));
        S[u * ldS + v] = make_float2(((u == v ? 3.f : 0.f) - g.x) * 0.5f, -g.y * 0.5f);
      }
      __syncthreads();
      for (int e = tid; e < tb2; e += nth) {
        const int u = e / tb, v = e % tb;
        float2 y = z;
        for (int k = 0; k < tb; ++k) y = add<float>(y, mul<float>(V[u * tb + k], S[k * ldS + v]));
        Vp[(size_t)par * tb2 + e] = y;
        if (t < a.log_rounds) a.logV[((size_t)t * 16 + me) * tb2 + e] = y;
      }
      if (tid == 0 && t < a.log_rounds) a.logB[(size_t)t * 16 + me] = P0 | (P1 << 16);
      cluster.sync();

      // (4) own columns X (N x 2b) <- X V, V the published (refined) copy:
      //     item (row i, half h) makes the outputs v = h b .. h b + b - 1 of
      //     row i (2N <= 768 items)
      {
        const float2* Vc = Vp + (size_t)par * tb2;
        const bool act = tid < 2 * N;
        const int i = act ? tid % N : 0, h = act ? tid / N : 0;
        float2 x[kBjMaxTb];
#pragma unroll
        for (int u = 0; u < kBjMaxTb; ++u) x[u] = (act && u < tb) ? col(u)[i] : z;
        __syncthreads();
        if (act) {
#pragma unroll
          for (int vv = 0; vv < kBjMaxB; ++vv) {
            if (vv < b) {
              const int v = h * b + vv;
              float2 y = z;
#pragma unroll
              for (int u = 0; u < kBjMaxTb; ++u)
                if (u < tb) y = add<float>(y, mul<float>(x[u], Vc[u * tb + v]));
              col(v)[i] = y;
            }
          }
        }
        __syncthreads();
      }
      // (5) for every pair d, rows L_d of the own columns <- V_d^H (rows L_d);
      //     V_d staged from CTA d kBjStage pairs at a time; item (pair dd of
      //     the stage, own column j, part hp of H) makes the outputs
      //     u = hp, hp + H, ... (H parts: as many items as there are threads)
      {
        const int H = min(tb, nth / (kBjStage * tb));
        for (int d0 = 0; d0 < 16; d0 += kBjStage) {
          for (int e = tid; e < kBjStage * tb2; e += nth) {
            const int dd = e / tb2, w = e - dd * tb2;
            const float2* src = cluster.map_shared_rank(Vp, d0 + dd);
            Vst[e] = src[(size_t)par * tb2 + w];
          }
          __syncthreads();
          const bool act = tid < kBjStage * tb * H;
          const int dd = act ? tid / (tb * H) : 0;
          const int rem = act ? tid - dd * tb * H : 0;
          const int j = rem % tb, hp = rem / tb;
          const int d = d0 + dd;
          const int Q0 = bj_player(d, r, 32), Q1 = bj_player(31 - d, r, 32);
          auto gd = [&](int k) { return k < b ? Q0 * b + k : Q1 * b + (k - b); };
          float2* xc = col(j);
          float2 x[kBjMaxTb];
#pragma unroll
          for (int k = 0; k < kBjMaxTb; ++k) x[k] = (act && k < tb) ? xc[gd(k)] : z;
          __syncthreads();
          if (act) {
            const float2* Vd = Vst + (size_t)dd * tb2;
            for (int u = hp; u < tb; u += H) {
              float2 y = z;
#pragma unroll
              for (int k = 0; k < kBjMaxTb; ++k)
                if (k < tb) y = add<float>(y, mulc<float>(x[k], Vd[k * tb + u]));  // conj(V_d[k][u]) x_k
              xc[gd(u)] = y;
            }
          }
          __syncthreads();
        }
      }
      // (6) last round of a sweep: max |A_ij| (i != j) of the own columns and
      //     max |A_ii|, published for the decision after the barrier
      if (r == 30) {
        float off = 0.f, dm = 0.f;
        for (int e = tid; e < tb * N; e += nth) {
          const int u = e / N, i = e - u * N;
          const int g = gl(u);
          if (g >= n || i >= n) continue;
          const float2 v = col(u)[i];
          const float m = sqrtf(v.x * v.x + v.y * v.y);
          if (i == g) dm = fmaxf(dm, m);
          else off = fmaxf(off, m);
        }
        for (int o = 16; o > 0; o >>= 1) {
          off = fmaxf(off, __shfl_xor_sync(0xffffffffu, off, o));
          dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
        }
        if (lane == 0) {
          red[4 + warp] = off;
          red[4 + 32 + warp] = dm;
        }
        __syncthreads();
        if (tid == 0) {
          float o2 = 0.f, d2 = 0.f;
          for (int w = 0; w < nwarps; ++w) {
            o2 = fmaxf(o2, red[4 + w]);
            d2 = fmaxf(d2, red[4 + 32 + w]);
          }
          red[2 * par] = o2;
          red[2 * par + 1] = d2;
        }
      }
      // (7) both blocks to the CTAs of their next positions (other parity)
      for (int s = 0; s < 2; ++s) {
        const int x = bj_next(s == 0 ? pos0 : pos1);
        const int dc = bj_pair(x), ds = x < 16 ? 0 : 1;
        float4* dst = (float4*)(cluster.map_shared_rank(blk, dc) + (size_t)(par ^ 1) * 2 * slotsz +
                                (size_t)ds * slotsz);
        const float4* src = (const float4*)(cur + (size_t)s * slotsz);
        for (size_t e = tid; e < slotsz / 2; e += nth) dst[e] = src[e];
      }
      cluster.sync();
      if (r == 30) {
        goff = 0.f;
        gdm = 0.f;
        for (int c = 0; c < kBjCluster; ++c) {
          const float* rr = cluster.map_shared_rank(red, c);
          goff = fmaxf(goff, rr[2 * par]);
          gdm = fmaxf(gdm, rr[2 * par + 1]);
        }
      }
    }
    ++sweep;
    if (goff <= a.tol * fmaxf(gdm, 1e-30f) || sweep >= a.max_sweeps) break;
  }

  // ---- results from the last round's own columns (still in place): the
  //      diagonal of the own indices, the sweeps and the rounds logged
  {
    const int rl = (t - 1) % 31;  // round index of the last round within its sweep
    const float2* last = blk + (size_t)((t - 1) & 1) * 2 * slotsz;
    const int P0 = bj_player(pos0, rl, 32), P1 = bj_player(pos1, rl, 32);
    for (int u = tid; u < tb; u += nth) {
      const int g = u < b ? P0 * b + u : P1 * b + (u - b);
      if (g < n) a.diag[g] = (double)last[(size_t)u * N + g].x;
    }
  }
  if (me == 0 && tid == 0) {
    a.info[0] = 0;
    a.info[1] = sweep;
    a.info[2] = t;
  }
  cluster.sync();
}

// Q = J_0 J_1 ... J_{R-1} from the logged V's (R = info[2] rounds): rows of Q
// evolve independently, q <- q J_t, i.e. q[L_d] <- q[L_d] V_{t,d} for every
// pair d.  A block holds kBjQRows rows in shared memory (rows of the identity
// at the start); item (row, pair, output u) a thread; the next round's column
// of V is fetched before the barrier that closes the current one.
constexpr int kBjQRows = 1;
__global__ void __launch_bounds__(384) k_bjacobi_qlog(const float2* __restrict__ logV,
                                                      const int* __restrict__ logB,
                                                      const int* __restrict__ info, int n, int b,
                                                      double2* __restrict__ Q, int64_t ldq) {
  extern __shared__ __align__(16) unsigned char qbsm[];
  const int N = 32 * b, tb = 2 * b, tb2 = tb * tb;
  float2* qs = (float2*)qbsm;  // [kBjQRows][N]
  const int i0 = blockIdx.x * kBjQRows;
  const int nr = min(kBjQRows, n - i0);
  for (int e = threadIdx.x; e < kBjQRows * N; e += blockDim.x) {
    const int r = e / N, c = e - r * N;
    qs[e] = make_float2((r < nr && i0 + r == c) ? 1.f : 0.f, 0.f);
  }
  const int R = info[2];
  const int it = threadIdx.x;
  const bool act = it < kBjQRows * 16 * tb;  // = kBjQRows N
  const int r = act ? it / (16 * tb) : 0;
  const int w = act ? it - r * 16 * tb : 0;
  const int d = w / tb, u = w - d * tb;
  float2 vc[kBjMaxTb];  // column u of V_{t,d}
  int bb = 0;
  if (act && R > 0) {
#pragma unroll
    for (int k = 0; k < kBjMaxTb; ++k)
      vc[k] = k < tb ? logV[(size_t)d * tb2 + (size_t)k * tb + u] : make_float2(0.f, 0.f);
    bb = logB[d];
  }
  __syncthreads();
  for (int rd = 0; rd < R; ++rd) {
    const int b0 = bb & 0xffff, b1 = bb >> 16;
    auto gd = [&](int k) { return k < b ? b0 * b + k : b1 * b + (k - b); };
    float2 y = make_float2(0.f, 0.f);
    if (act) {
      const float2* row = qs + (size_t)r * N;
#pragma unroll
      for (int k = 0; k < kBjMaxTb; ++k)
        if (k < tb) y = add<float>(y, mul<float>(row[gd(k)], vc[k]));
    }
    // next round's column of V while the others finish reading
    if (act && rd + 1 < R) {
      const size_t base = ((size_t)(rd + 1) * 16 + d) * tb2;
#pragma unroll
      for (int k = 0; k < kBjMaxTb; ++k)
        if (k < tb) vc[k] = logV[base + (size_t)k * tb + u];
    }
    const int wpos = act ? gd(u) : 0;
    if (act && rd + 1 < R) bb = logB[(size_t)(rd + 1) * 16 + d];
    __syncthreads();
    if (act) qs[(size_t)r * N + wpos] = y;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
    const int c = e / nr, rr = e - c * nr;
    const float2 v = qs[(size_t)rr * N + c];
    Q[(size_t)c * ldq + i0 + rr] = make_double2((double)v.x, (double)v.y);
  }
}

bool jacobi32_block_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("PWH_JACOBI_BLOCK");
    return e && e[0] == '1';
  }();
  return on;
}

size_t jacobi32_block_log_bytes(int n, int max_sweeps) {
  const int b = (n + 31) / 32, tb = 2 * b;
  const size_t rounds = (size_t)max_sweeps * 31;
  return rounds * 16 * ((size_t)tb * tb * sizeof(float2) + sizeof(int)) + 256;
}

bool jacobi32_block(System& s, DenseWs& w, const double2* A, int64_t lda, int n, double tol,
                    int max_sweeps, double2* Q, int64_t ldq, double* diag, int* info,
                    cudaStream_t st) {
  (void)s;
  if (n < 64 || n > 32 * kBjMaxB) return false;
  const int b = (n + 31) / 32, N = 32 * b, tb = 2 * b;
  const size_t smem = bj_smem_bytes(b);
  if (smem > 227 * 1024) return false;
  static std::once_flag attr_once;
  static bool attr_ok = false;
  std::call_once(attr_once, [] {
    attr_ok = cudaFuncSetAttribute(k_bjacobi_dsm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   227 * 1024) == cudaSuccess &&
              cudaFuncSetAttribute(k_bjacobi_dsm, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                   1) == cudaSuccess;
    cudaGetLastError();
  });
  if (!attr_ok) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kBjCluster);
  cfg.blockDim = dim3(kBjThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kBjCluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  {
    static std::mutex mu;
    static size_t fits_upto = 0, fails_from = ~size_t(0);
    std::lock_guard<std::mutex> lock(mu);
    if (smem > fits_upto) {
      if (smem >= fails_from) return false;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, (void*)k_bjacobi_dsm, &cfg) != cudaSuccess ||
          nclusters < 1) {
        cudaGetLastError();
        fails_from = smem;
        return false;
      }
      fits_upto = smem;
    }
  }
  ensure(w.jlog, jacobi32_block_log_bytes(n, max_sweeps));
  BjArgs a;
  a.A = A;
  a.lda = lda;
  a.diag = diag;
  a.info = info;
  a.log_rounds = (int64_t)max_sweeps * 31;
  a.logV = (float2*)w.jlog.p;
  a.logB = (int*)(a.logV + (size_t)a.log_rounds * 16 * tb * tb);
  a.n = n;
  a.b = b;
  a.max_sweeps = max_sweeps;
  a.tol = (float)tol;
  PWH_CUDA(cudaLaunchKernelEx(&cfg, k_bjacobi_dsm, a));
  note_launch();
  k_bjacobi_qlog<<<(n + kBjQRows - 1) / kBjQRows, kBjQRows * N, (size_t)kBjQRows * N * sizeof(float2), st>>>(
      a.logV, a.logB, info, n, b, Q, ldq);
  PWH_LAUNCH_CHECK();
  return true;
}

}  // namespace pwh
