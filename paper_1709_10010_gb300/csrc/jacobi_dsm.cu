// FP32 parallel cyclic Jacobi with the whole matrix resident in the shared
// memory of one thread-block cluster (16 CTAs on one GPC), for the subspace
// diagonalisation of the block Davidson method (Sec. "New parallelization
// levels": the O_ij = <psi_i|O|psi_j> matrices and their diagonalization).
//
// The same two-sided complex Jacobi as k_jacobi (round-robin pairing, np - 1
// rounds a sweep, every round rotates np/2 disjoint pairs), distributed by
// column pairs instead of through global memory:
//
//  * tournament positions 0..np-1: pair k plays positions k and np-1-k; CTA c
//    owns pairs [c PP, c PP + PP) and keeps, for each of its positions, the
//    full column of A and of Q (rows in original index order) of the index
//    ("player") standing there.  Between rounds every player except the one
//    at position 0 steps to the next position (np-1 wraps to 1); only the
//    players crossing to a neighbouring CTA move data (at most two columns of
//    A and two of Q per CTA and round, written into the neighbour's inbox
//    through distributed shared memory), the rest move by table update.
//  * the diagonal is replicated in every CTA: all CTAs apply every round's
//    2 x 2 diagonal updates from the published (c, s, A_pq) identically.
//  * a round, between two cluster barriers: land the arrivals of the last
//    step, read all np/2 rotations of the round (published by their owners
//    before the barrier), apply J^H A J to the own columns (2 x 2 blocks: row
//    pair x own column pair, in place) and Q J to the own Q columns, update
//    the diagonal, send the departing columns, then compute and publish the
//    next round's rotations of the own pairs (A_pq from whichever of the two
//    columns stays here).  Rotation tables and inboxes alternate between two
//    copies by round parity, so one barrier a round suffices.
//  * at the end of each sweep every CTA publishes max |A_ij| (i != j) of its
//    columns and max |A_ii|; all CTAs take the same decision from the same
//    numbers, so the control flow stays uniform and every barrier is met.
//
// No software spin anywhere: only the hardware cluster barrier.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "common.cuh"
#include "dense.cuh"
#include "jacobi_rot.cuh"

namespace cg = cooperative_groups;

namespace pwh {

constexpr int kDsmCluster = 16;
constexpr int kDsmThreads = 1024;

struct JdsmArgs {
  const double2* A;  // n x n Hermitian start (full), ld lda
  int64_t lda;
  double* diag;      // out: final diagonal (eigenvalue estimates), n
  int* info;         // out: [0] = 0, [1] = sweeps used, [2] = rounds logged
  float4* log;       // out: rotations, round t pair k at [t P + k]: (s, c, p | q << 16)
  int64_t log_rounds;  // capacity of log in rounds
  int n, np, P, PP, max_sweeps;
  float tol;
};

// shared-memory layout of one CTA, in this order:
//   float2 colA[nbuf n]                    column buffers, nbuf = 2 PP + 4 (the
//                                          last four: inboxes [parity][side])
//   float4 rot[2][PP][2]                   published rotations of the own pairs,
//                                          by round parity: (s, c, p | q << 16),
//                                          (A_pq, -, -)
//   float4 allr[P][2]                      the round's rotations of every pair
//   float  dg[np]                          the diagonal, replicated in every CTA
//   float  red[66]                         [0] off, [1] dmax (published), partials
//   int    bufof[2 PP], nbufof[2 PP]       buffer of each own slot (current, next)
//   int    own[4][PP]                      the round's p, q, buffer(p), buffer(q)
__host__ __device__ inline size_t jdsm_smem_bytes(int n, int P, int PP) {
  const size_t nbuf = 2 * (size_t)PP + 4;
  const int np = 2 * P;
  return nbuf * n * sizeof(float2) + (4 * (size_t)PP + 2 * (size_t)P) * sizeof(float4) +
         (size_t)(np + 66) * sizeof(float) + (size_t)(8 * PP) * sizeof(int);
}

// position -> pair; previous and next position of the round-robin (every
// position but 0 steps forward, np-1 wraps to 1)
__device__ __forceinline__ int jd_pair(int x, int np, int P) { return x < P ? x : np - 1 - x; }
__device__ __forceinline__ int jd_prev(int x, int np) { return x == 0 ? 0 : (x == 1 ? np - 1 : x - 1); }
__device__ __forceinline__ int jd_next(int x, int np) { return x == 0 ? 0 : (x == np - 1 ? 1 : x + 1); }
// index standing at position x in round r of a sweep (position x holds x at r = 0)
__device__ __forceinline__ int jd_player(int x, int r, int np) {
  return x == 0 ? 0 : 1 + (x - 1 - r + (np - 1)) % (np - 1);
}

__global__ void __launch_bounds__(kDsmThreads, 1) k_jacobi_dsm(JdsmArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char dsm[];
  const int n = a.n, np = a.np, P = a.P, PP = a.PP;
  const int me = (int)cluster.block_rank();
  const int k0 = me * PP;
  const int ns = max(0, min(PP, P - k0));  // own pairs
  const int nslot = 2 * ns;
  const int nbuf = 2 * PP + 4;
  const int ibuf0 = 2 * PP;  // inbox buffer ibuf0 + 2 parity + side
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  float2* colA = (float2*)dsm;
  float4* rot = (float4*)(colA + (size_t)nbuf * n);
  float4* allr = rot + 4 * PP;
  float* dg = (float*)(allr + 2 * P);
  float* red = dg + np;
  int* bufof = (int*)(red + 66);
  int* nbufof = bufof + 2 * PP;
  int* own = nbufof + 2 * PP;  // own[0..PP) p, [PP..2PP) q, then buffers of p and q

  // Fixed per CTA: own slot s stands at position pos(s) (pair k0 + s/2, first
  // or second place); the slots whose index leaves for a neighbouring CTA at
  // each step and the slots filled from an inbox.  At most one of each per
  // side, and (for at least two pairs per CTA) never both places of a pair.
  auto pos_of = [&](int s) { const int k = k0 + (s >> 1); return (s & 1) ? np - 1 - k : k; };
  auto slot_of = [&](int x) { const int k = jd_pair(x, np, P); return 2 * (k - k0) + (x >= P ? 1 : 0); };
  int n_out = 0, out_slot[2] = {-1, -1}, out_cta[2] = {0, 0}, out_box[2] = {0, 0};
  int n_in = 0, in_slot[2] = {-1, -1}, in_box[2] = {0, 0};
  for (int s = 0; s < nslot; ++s) {
    const int x = pos_of(s);
    const int d = jd_next(x, np);
    const int od = jd_pair(d, np, P) / PP;
    if (od != me && n_out < 2) {
      out_slot[n_out] = s;
      out_cta[n_out] = od;
      out_box[n_out] = d < P ? 0 : 1;
      ++n_out;
    }
    const int src = jd_prev(x, np);
    if (jd_pair(src, np, P) / PP != me && n_in < 2) {
      in_slot[n_in] = s;
      in_box[n_in] = x < P ? 0 : 1;
      ++n_in;
    }
  }

  // Rotations of round r for the own pairs into rot[par]: A_pq from whichever
  // of the two columns is here (an arriving column is still in an inbox when
  // pending), the diagonal from the replicated copy.
  auto publish = [&](int r, int par, bool pending, int64_t tr) {
    for (int j = threadIdx.x; j < ns; j += blockDim.x) {
      int p = jd_player(pos_of(2 * j), r, np), q = jd_player(pos_of(2 * j + 1), r, np);
      int bp = bufof[2 * j], bq = bufof[2 * j + 1];
      bool hp = true, hq = true;
      if (pending) {
        for (int i = 0; i < n_in; ++i) {
          if (in_slot[i] == 2 * j) hp = false;
          if (in_slot[i] == 2 * j + 1) hq = false;
        }
      }
      if (p > q) {
        int t = p; p = q; q = t;
        t = bp; bp = bq; bq = t;
        const bool h = hp; hp = hq; hq = h;
      }
      float c = 1.f;
      float2 sv = make_float2(0.f, 0.f), apq = make_float2(0.f, 0.f);
      if (q < n) {
        if (hq) {
          apq = colA[(size_t)bq * n + p];
        } else {
          const float2 v = colA[(size_t)bp * n + q];
          apq = make_float2(v.x, -v.y);
        }
        jacobi_rotation_fast(apq, dg[p], dg[q], c, sv);
      }
      const float4 r0 = make_float4(sv.x, sv.y, c, __int_as_float(p | (q << 16)));
      rot[(par * PP + j) * 2] = r0;
      if (tr < a.log_rounds) a.log[tr * P + k0 + j] = r0;
      rot[(par * PP + j) * 2 + 1] = make_float4(apq.x, apq.y, 0.f, 0.f);
    }
  };
  // Arrivals of the last step: inbox[par] into the buffers the tables gave them.
  auto land = [&](int r, int par) {
    for (int i = 0; i < n_in; ++i) {
      const int b = bufof[in_slot[i]];
      const size_t src = (size_t)(ibuf0 + 2 * par + in_box[i]) * n;
      if (jd_player(pos_of(in_slot[i]), r, np) < n) {
        for (int e = threadIdx.x; e < n; e += blockDim.x) colA[(size_t)b * n + e] = colA[src + e];
      }
    }
  };

  // ---- load: position x starts with index x
  for (int s = threadIdx.x; s < nslot; s += blockDim.x) bufof[s] = s;
  for (int i = threadIdx.x; i < np; i += blockDim.x) dg[i] = i < n ? (float)a.A[(size_t)i * a.lda + i].x : 0.f;
  for (int t = threadIdx.x; t < nslot * n; t += blockDim.x) {
    const int s = t / n, i = t - s * n;
    const int pl = pos_of(s);
    if (pl < n) {
      const double2 v = a.A[(size_t)pl * a.lda + i];
      colA[(size_t)s * n + i] = make_float2((float)v.x, (float)v.y);
    }
  }
  __syncthreads();
  publish(0, 0, false, 0);
  cluster.sync();

  // warp tasks of the update: chunks of 64 row pairs per own column pair; a
  // warp's next task is nwarps further on
  const int nchA = (P + 63) >> 6;
  const int stepA_j = nwarps / nchA, stepA_c = nwarps - stepA_j * nchA;
  const float2 z = make_float2(0.f, 0.f);
  int sweep = 0, t = 0;  // t: rounds done (its parity picks the rotation table and inboxes)
  while (true) {
    for (int r = 0; r < np - 1; ++r, ++t) {
      const int par = t & 1;
      // (1) every rotation of the round from the CTAs that own them (remote
      //     loads issued first), the arrivals of the last step into their
      //     buffers meanwhile, then the indices and buffers of the own pairs
      float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0;
      if (threadIdx.x < P) {
        const int o = threadIdx.x / PP, jj = threadIdx.x - o * PP;
        const float4* src = cluster.map_shared_rank(rot, o) + (par * PP + jj) * 2;
        g0 = src[0];
        g1 = src[1];
      }
      if (t > 0) land(r, par);
      if (threadIdx.x < P) {
        allr[2 * threadIdx.x] = g0;
        allr[2 * threadIdx.x + 1] = g1;
      }
      for (int i = threadIdx.x + blockDim.x; i < P; i += blockDim.x) {
        const int o = i / PP, jj = i - o * PP;
        const float4* src = cluster.map_shared_rank(rot, o) + (par * PP + jj) * 2;
        allr[2 * i] = src[0];
        allr[2 * i + 1] = src[1];
      }
      for (int j = threadIdx.x; j < ns; j += blockDim.x) {
        int p = jd_player(pos_of(2 * j), r, np), q = jd_player(pos_of(2 * j + 1), r, np);
        int bp = bufof[2 * j], bq = bufof[2 * j + 1];
        if (p > q) {
          int u = p; p = q; q = u;
          u = bp; bp = bq; bq = u;
        }
        own[j] = p;
        own[PP + j] = q;
        own[2 * PP + j] = bp;
        own[3 * PP + j] = bq;
      }
      __syncthreads();
      // (2) A <- J^H A J on the own columns: a warp task is one own column
      //     pair against 64 row pairs (two 2 x 2 blocks a lane); the pair
      //     element of an own pair becomes zero, its diagonal lives in dg.
      //     Tasks are dealt to warps round-robin: (j, chunk) advance by
      //     nwarps without division.  (Q is accumulated afterwards from the
      //     rotation log, k_jacobi_qlog.)
      {
        const int ntA = ns * nchA;
        int j = warp / nchA, c = warp - (warp / nchA) * nchA;
        for (int task = warp; task < ntA; task += nwarps) {
          const float4 Rl = allr[2 * (k0 + j)];
          const float cl = Rl.z;
          const float2 sl = make_float2(Rl.x, Rl.y);
          const int ql = own[PP + j];
          const bool vl = ql < n;
          float2* cp = colA + (size_t)own[2 * PP + j] * n;
          float2* cq = colA + (size_t)own[3 * PP + j] * n;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int kk = c * 64 + h * 32 + lane;
            if (kk < P) {
              const float4 Rk = allr[2 * kk];
              const int pqk = __float_as_int(Rk.w);
              const int pk = pqk & 0xffff, qk = pqk >> 16;
              const bool vk = qk < n;
              if (kk == k0 + j) {
                if (vk) {
                  cq[pk] = z;
                  cp[qk] = z;
                }
              } else {
                const float2 a00 = cp[pk];
                const float2 a01 = vl ? cq[pk] : z;
                const float2 a10 = vk ? cp[qk] : z;
                const float2 a11 = (vk && vl) ? cq[qk] : z;
                float2 y00, y01, y10, y11;
                jacobi_block<float>(a00, a01, a10, a11, Rk.z, make_float2(Rk.x, Rk.y), cl, sl, y00,
                                    y01, y10, y11);
                cp[pk] = y00;
                if (vl) cq[pk] = y01;
                if (vk) cp[qk] = y10;
                if (vk && vl) cq[qk] = y11;
              }
            }
          }
          c += stepA_c;
          j += stepA_j;
          if (c >= nchA) {
            c -= nchA;
            ++j;
          }
        }
      }
      // the diagonal of every rotated pair (each CTA, identically)
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const float4 R0 = allr[2 * i], R1 = allr[2 * i + 1];
        const int pq = __float_as_int(R0.w);
        const int p = pq & 0xffff, q = pq >> 16;
        if (q >= n) continue;
        const float2 sv = make_float2(R0.x, R0.y), apq = make_float2(R1.x, R1.y);
        float2 y00, y01, y10, y11;
        jacobi_block<float>(make_float2(dg[p], 0.f), apq, make_float2(apq.x, -apq.y),
                            make_float2(dg[q], 0.f), R0.z, sv, R0.z, sv, y00, y01, y10, y11);
        dg[p] = y00.x;
        dg[q] = y11.x;
      }
      __syncthreads();
      // (3b) last round of a sweep: max |A_ij| (i != j) of the own columns and
      //      max |A_ii|, published for the decision after the barrier
      if (r == np - 2) {
        float off = 0.f, dm = 0.f;
        for (int e = threadIdx.x; e < nslot * n; e += blockDim.x) {
          const int sl = e / n, i = e - sl * n;
          const int pl = jd_player(pos_of(sl), r, np);
          if (pl >= n || i == pl) continue;
          const float2 v = colA[(size_t)bufof[sl] * n + i];
          off = fmaxf(off, sqrtf(v.x * v.x + v.y * v.y));
        }
        for (int i = threadIdx.x; i < n; i += blockDim.x) dm = fmaxf(dm, fabsf(dg[i]));
        for (int o = 16; o > 0; o >>= 1) {
          off = fmaxf(off, __shfl_xor_sync(0xffffffffu, off, o));
          dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
        }
        if (lane == 0) {
          red[2 + warp] = off;
          red[34 + warp] = dm;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          float o2 = 0.f, d2 = 0.f;
          for (int w = 0; w < nwarps; ++w) {
            o2 = fmaxf(o2, red[2 + w]);
            d2 = fmaxf(d2, red[34 + w]);
          }
          red[0] = o2;
          red[1] = d2;
        }
      }
      // (4) buffers after the step: indices that stay here keep theirs, the
      //     arrivals take those of the departures
      for (int sl = threadIdx.x; sl < nslot; sl += blockDim.x) {
        const int src = jd_prev(pos_of(sl), np);
        if (jd_pair(src, np, P) / PP == me) nbufof[sl] = bufof[slot_of(src)];
      }
      if (threadIdx.x == 0)
        for (int i = 0; i < n_in; ++i) nbufof[in_slot[i]] = bufof[out_slot[i]];
      // (5) departing columns into the neighbours' inboxes of the other parity
      for (int o = 0; o < n_out; ++o) {
        if (jd_player(pos_of(out_slot[o]), r, np) >= n) continue;
        const int b = bufof[out_slot[o]];
        const size_t dst = (size_t)(ibuf0 + 2 * (par ^ 1) + out_box[o]) * n;
        float2* rA = cluster.map_shared_rank(colA, out_cta[o]) + dst;
        for (int i = threadIdx.x; i < n; i += blockDim.x) rA[i] = colA[(size_t)b * n + i];
      }
      __syncthreads();
      {
        int* u = bufof; bufof = nbufof; nbufof = u;
      }
      // (6) rotations of the next round (arrivals still in their inboxes)
      publish(r + 1 == np - 1 ? 0 : r + 1, par ^ 1, true, (int64_t)t + 1);
      cluster.sync();
    }
    ++sweep;
    float goff = 0.f, gdm = 0.f;
    for (int c = 0; c < (int)cluster.num_blocks(); ++c) {
      const float* rr = cluster.map_shared_rank(red, c);
      goff = fmaxf(goff, rr[0]);
      gdm = fmaxf(gdm, rr[1]);
    }
    if (goff <= a.tol * fmaxf(gdm, 1e-30f) || sweep >= a.max_sweeps) break;
  }

  // ---- results: the diagonal, the sweeps and the rounds logged (t)
  if (me == 0) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) a.diag[i] = (double)dg[i];
    if (threadIdx.x == 0) {
      a.info[0] = 0;
      a.info[1] = sweep;
      a.info[2] = t;
    }
  }
  cluster.sync();
}

// Q = J_0 J_1 ... J_{R-1} from the rotation log (R = info[2] rounds): rows of
// Q evolve independently, so each block takes kQlogRows rows in shared memory
// (starting as rows of the identity) and applies every round to them in
// order, a thread per (row, pair); the next round's rotation is fetched
// before the barrier that closes the current one.
constexpr int kQlogRows = 4;
__global__ void __launch_bounds__(1024) k_jacobi_qlog(const float4* __restrict__ log,
                                                      const int* __restrict__ info, int n, int P,
                                                      double2* __restrict__ Q, int64_t ldq) {
  extern __shared__ __align__(16) unsigned char qsm[];
  float2* qs = (float2*)qsm;  // [kQlogRows][n]
  const int i0 = blockIdx.x * kQlogRows;
  const int nr = min(kQlogRows, n - i0);
  for (int t = threadIdx.x; t < kQlogRows * n; t += blockDim.x) {
    const int r = t / n, c = t - r * n;
    qs[t] = make_float2((r < nr && i0 + r == c) ? 1.f : 0.f, 0.f);
  }
  const int R = info[2];
  const int it = threadIdx.x;  // one (row, pair) item a thread
  const bool active = it < kQlogRows * P;
  const int k = active ? it % P : 0, r = active ? it / P : 0;
  float4 rc = (active && R > 0) ? log[k] : make_float4(0.f, 0.f, 1.f, 0.f);
  __syncthreads();
  for (int rd = 0; rd < R; ++rd) {
    const float4 cur = rc;
    if (active && rd + 1 < R) rc = log[(size_t)(rd + 1) * P + k];
    if (active && r < nr) {
      const int pq = __float_as_int(cur.w);
      const int p = pq & 0xffff, q = pq >> 16;
      if (q < n) {
        const float c = cur.z;
        const float2 sv = make_float2(cur.x, cur.y);
        float2* row = qs + (size_t)r * n;
        const float2 q0 = row[p], q1 = row[q];
        row[p] = add<float>(scl<float>(q0, c), mul<float>(q1, make_float2(-sv.x, sv.y)));
        row[q] = add<float>(mul<float>(q0, sv), scl<float>(q1, c));
      }
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nr * n; t += blockDim.x) {
    const int c = t / nr, rr = t - c * nr;
    const float2 v = qs[(size_t)rr * n + c];
    Q[(size_t)c * ldq + i0 + rr] = make_double2((double)v.x, (double)v.y);
  }
}

size_t jacobi32_log_bytes(int n, int max_sweeps) {
  const int np = n + (n & 1);
  return (size_t)max_sweeps * (np - 1) * (np / 2) * sizeof(float4);
}

bool jacobi32_cluster(System& s, DenseWs& w, const double2* A, int64_t lda, int n, double tol,
                      int max_sweeps, double2* Q, int64_t ldq, double* diag, int* info,
                      cudaStream_t st) {
  (void)s;
  if (n < 64) return false;  // at least two pairs per CTA
  const int np = n + (n & 1), P = np / 2;
  const int PP = (P + kDsmCluster - 1) / kDsmCluster;
  const size_t smem = jdsm_smem_bytes(n, P, PP);
  if (smem > 220 * 1024 || n > 512) return false;  // k_jacobi_qlog: a thread per (row, pair)
  static std::once_flag attr_once;
  static bool attr_ok = false;
  std::call_once(attr_once, [] {
    attr_ok = cudaFuncSetAttribute(k_jacobi_dsm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   227 * 1024) == cudaSuccess &&
              cudaFuncSetAttribute(k_jacobi_dsm, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                  cudaSuccess;
    cudaGetLastError();
  });
  if (!attr_ok) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kDsmCluster);
  cfg.blockDim = dim3(kDsmThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kDsmCluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // can one cluster of this size and shared memory be resident?  (cached per size)
  {
    static std::mutex mu;
    static size_t fits_upto = 0, fails_from = ~size_t(0);
    std::lock_guard<std::mutex> lock(mu);
    if (smem > fits_upto) {
      if (smem >= fails_from) return false;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, (void*)k_jacobi_dsm, &cfg) != cudaSuccess ||
          nclusters < 1) {
        cudaGetLastError();
        fails_from = smem;
        return false;
      }
      fits_upto = smem;
    }
  }
  ensure(w.jlog, jacobi32_log_bytes(n, max_sweeps));
  JdsmArgs a;
  a.A = A; a.lda = lda; a.diag = diag; a.info = info;
  a.log = (float4*)w.jlog.p;
  a.log_rounds = (int64_t)max_sweeps * (np - 1);
  a.n = n; a.np = np; a.P = P; a.PP = PP; a.max_sweeps = max_sweeps; a.tol = (float)tol;
  PWH_CUDA(cudaLaunchKernelEx(&cfg, k_jacobi_dsm, a));
  note_launch();
  // eigenvectors from the logged rotations, rows spread over the GPU
  static std::once_flag q_once;
  std::call_once(q_once, [] {
    cudaFuncSetAttribute(k_jacobi_qlog, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  k_jacobi_qlog<<<(n + kQlogRows - 1) / kQlogRows, 1024, (size_t)kQlogRows * n * sizeof(float2), st>>>(
      a.log, info, n, P, Q, ldq);
  PWH_LAUNCH_CHECK();
  return true;
}

}  // namespace pwh
