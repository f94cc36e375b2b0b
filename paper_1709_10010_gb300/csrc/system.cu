// System set-up of libpwh: the plane-wave sphere and its orderings, the
// z-stick decomposition for the FFT passes, and the uploads of V_LOC, beta, D.
//
// Basis: {G : 1/2|k+G|^2 <= ecut} with q = sum_i (m_i + k_i) b_i evaluated in
// FP64 from the integer Miller indices, inclusive with a relative slack of
// 1e-12 for plane waves lying exactly on the cutoff (plane-wave coefficients c_{k,n}(G),
// Sec. "New parallelization levels").  Public order: ascending |k+G|^2, equal
// shells (relative 1e-10) ordered lexicographically by (m1, m2, m3) — the
// reproducible ordering asked for in Sec. "Large-record data file format".
// Internal order: lexicographic (m1, m2, m3), so that every z-stick (fixed
// m1, m2) is a contiguous run and sticks sharing m1 form one x-column.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>

#include "common.cuh"

namespace pwh {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;  // this thread's launches
void note_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
void note_launches(long long n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  t_launches += n;
}
long long launch_counter() { return t_launches; }

const char* const kKernelFamilyName[KF_COUNT] = {
    "fft_z_inverse_fp64", "fft_plane_fp64", "fft_z_forward_fp64", "fft_z_inverse_fp32",
    "fft_plane_fp32", "fft_z_forward_fp32", "tc_gemm_becp", "tc_gemm_backproj", "cgemm_fp64",
    "cgemm_fp32", "jacobi_fp64", "cholqr_fp64", "jacobi_fp32", "zgemm_fp64_tc", "zgemm_fp32_tc"};

cudaEvent_t KernelTimer::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void KernelTimer::resolve() {
  for (auto& p : pending) {
    float t = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
      ms[p.fam] += t;
      n[p.fam] += 1;
    }
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
}

void KernelTimer::reset() {
  resolve();
  for (int i = 0; i < KF_COUNT; ++i) {
    ms[i] = 0;
    n[i] = 0;
    flops[i] = 0;
    bytes[i] = 0;
  }
}

KernelTimer::~KernelTimer() {
  for (auto& p : pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : pool) cudaEventDestroy(e);
}

System::~System() {
  if (stream) cudaStreamSynchronize(stream);
  free_davidson_ws(dav);
  void* ptrs[] = {d_int_to_pub, d_kin, d_stick_off, d_stick_of, d_zpos, d_stick_col,
                  d_stick_y, d_col_x, d_stick_at, d_xcol, d_tw64, d_tw32, d_twdf, d_perm, d_v64, d_v32, d_vdf, d_beta64,
                  d_ddiag, d_dfull, d_beta32, d_beta_bf16, d_beta_bf16_t,
                  ws_fft.p, ws_vnl.p, ws_grid.p, ws_tune.p, ws_psi.p, ws_hpsi.p, ws_becp.p, ws_split.p, ws_host.p,
                  ws_tc.p, ws_oz.p, d_err, d_shell, d_Tshell, d_mlp, d_gam_pos,
                  d_boxidx, d_kern, d_ace, ws_ace.p, d_q, d_ksq, ws_ov.p};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

static bool smooth235(int n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

static int smooth_even_at_least(int n) {
  int m = std::max(n, 2);
  while (!(m % 2 == 0 && smooth235(m))) ++m;
  return m;
}

static int imod(int a, int n) { return ((a % n) + n) % n; }

static void build_basis(System& s, const int fft_req[3]) {
  const double* A = s.lattice;
  double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
               A[2] * (A[3] * A[7] - A[4] * A[6]);
  PWH_CHECK_ARG(std::isfinite(det) && std::fabs(det) > 1e-12, "lattice is singular");
  // b_i = 2 pi (a_j x a_k) / det, rows of the reciprocal basis
  double B[9];
  const double tp = 2.0 * M_PI;
  for (int i = 0; i < 3; ++i) {
    const double* aj = A + 3 * ((i + 1) % 3);
    const double* ak = A + 3 * ((i + 2) % 3);
    B[3 * i + 0] = tp * (aj[1] * ak[2] - aj[2] * ak[1]) / det;
    B[3 * i + 1] = tp * (aj[2] * ak[0] - aj[0] * ak[2]) / det;
    B[3 * i + 2] = tp * (aj[0] * ak[1] - aj[1] * ak[0]) / det;
  }
  const double gc = std::sqrt(2.0 * s.ecut);
  int bound[3];
  for (int i = 0; i < 3; ++i) {
    double an = std::sqrt(A[3 * i] * A[3 * i] + A[3 * i + 1] * A[3 * i + 1] +
                          A[3 * i + 2] * A[3 * i + 2]);
    bound[i] = (int)std::floor(gc * an / tp + std::fabs(s.kpoint[i])) + 1;
    PWH_CHECK_ARG(bound[i] < 2000, "cutoff too large for the cell");
  }
  struct PW { int m[3]; double q2; int64_t shell; };
  std::vector<PW> pw;
  for (int a = -bound[0]; a <= bound[0]; ++a)
    for (int b = -bound[1]; b <= bound[1]; ++b)
      for (int c = -bound[2]; c <= bound[2]; ++c) {
        double f0 = a + s.kpoint[0], f1 = b + s.kpoint[1], f2 = c + s.kpoint[2];
        double qx = f0 * B[0] + f1 * B[3] + f2 * B[6];
        double qy = f0 * B[1] + f1 * B[4] + f2 * B[7];
        double qz = f0 * B[2] + f1 * B[5] + f2 * B[8];
        double q2 = qx * qx + qy * qy + qz * qz;
        if (0.5 * q2 <= s.ecut * (1.0 + 1e-12)) pw.push_back(PW{{a, b, c}, q2, 0});
      }
  PWH_CHECK_ARG(!pw.empty(), "empty plane-wave sphere");
  PWH_CHECK_ARG(pw.size() < (size_t)INT32_MAX / 4, "too many plane waves");
  auto lex = [](const PW& x, const PW& y) {
    if (x.m[0] != y.m[0]) return x.m[0] < y.m[0];
    if (x.m[1] != y.m[1]) return x.m[1] < y.m[1];
    return x.m[2] < y.m[2];
  };
  std::sort(pw.begin(), pw.end(), [&](const PW& x, const PW& y) {
    if (x.q2 != y.q2) return x.q2 < y.q2;
    return lex(x, y);
  });
  int64_t sh = 0;
  for (size_t j = 0; j < pw.size(); ++j) {
    if (j > 0 && (pw[j].q2 - pw[j - 1].q2) > 1e-10 * pw[j].q2) ++sh;
    pw[j].shell = sh;
  }
  std::stable_sort(pw.begin(), pw.end(), [&](const PW& x, const PW& y) {
    if (x.shell != y.shell) return x.shell < y.shell;
    return lex(x, y);
  });
  s.npw = (int64_t)pw.size();
  s.miller.resize(3 * s.npw);
  s.kin_pub.resize(s.npw);
  s.shell_pub.resize(s.npw);
  s.Tshell_h.clear();
  for (int64_t j = 0; j < s.npw; ++j) {
    s.shell_pub[j] = (int32_t)pw[j].shell;
    if ((int64_t)s.Tshell_h.size() <= pw[j].shell) s.Tshell_h.push_back(0.5 * pw[j].q2);
  }
  s.nshell = (int)s.Tshell_h.size();
  int mmax[3] = {0, 0, 0};
  for (int64_t j = 0; j < s.npw; ++j) {
    for (int d = 0; d < 3; ++d) {
      s.miller[3 * j + d] = pw[j].m[d];
      mmax[d] = std::max(mmax[d], std::abs(pw[j].m[d]));
    }
    s.kin_pub[j] = 0.5 * pw[j].q2;
  }
  int n[3];
  for (int d = 0; d < 3; ++d) {
    if (fft_req[d] == 0) {
      n[d] = smooth_even_at_least(4 * mmax[d] + 1);
    } else {
      PWH_CHECK_ARG(smooth235(fft_req[d]), "FFT size must be 2,3,5-smooth");
      PWH_CHECK_ARG(fft_req[d] >= 2 * mmax[d] + 1, "FFT size below 2*mmax+1");
      n[d] = fft_req[d];
    }
    PWH_CHECK_ARG(n[d] <= kMaxFft, "FFT size above 512");
  }
  s.n1 = n[0]; s.n2 = n[1]; s.n3 = n[2];

  // internal order: lexicographic (m1, m2, m3)
  std::vector<int32_t> order(s.npw);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
    const int32_t* a = &s.miller[3 * (int64_t)x];
    const int32_t* b = &s.miller[3 * (int64_t)y];
    if (a[0] != b[0]) return a[0] < b[0];
    if (a[1] != b[1]) return a[1] < b[1];
    return a[2] < b[2];
  });
  s.int_to_pub = order;
  s.stick_off.clear(); s.stick_col.clear(); s.stick_y.clear(); s.col_x.clear();
  int prev1 = INT32_MIN, prev2 = INT32_MIN;
  for (int64_t i = 0; i < s.npw; ++i) {
    const int32_t* m = &s.miller[3 * (int64_t)order[i]];
    if (m[0] != prev1) {
      s.col_x.push_back(imod(m[0], s.n1));
      prev2 = INT32_MIN;
    }
    if (m[0] != prev1 || m[1] != prev2) {
      s.stick_off.push_back((int32_t)i);
      s.stick_col.push_back((int32_t)s.col_x.size() - 1);
      s.stick_y.push_back(imod(m[1], s.n2));
    }
    prev1 = m[0];
    prev2 = m[1];
  }
  s.stick_off.push_back((int32_t)s.npw);
  s.nsticks = (int)s.stick_col.size();
  s.ncols = (int)s.col_x.size();
}

template <typename T> static T* upload(const std::vector<T>& v, cudaStream_t st) {
  T* p = nullptr;
  PWH_CUDA(cudaMalloc((void**)&p, std::max<size_t>(1, v.size()) * sizeof(T)));
  if (!v.empty())
    PWH_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return p;
}

static void upload_basis(System& s) {
  cudaStream_t st = s.stream;
  s.d_int_to_pub = upload(s.int_to_pub, st);
  std::vector<double> kin(s.npw);
  std::vector<int32_t> stick_of(s.npw);
  std::vector<int16_t> zpos(s.npw);
  for (int st_i = 0; st_i < s.nsticks; ++st_i)
    for (int i = s.stick_off[st_i]; i < s.stick_off[st_i + 1]; ++i) stick_of[i] = st_i;
  for (int64_t i = 0; i < s.npw; ++i) {
    kin[i] = s.kin_pub[s.int_to_pub[i]];
    zpos[i] = (int16_t)imod(s.miller[3 * (int64_t)s.int_to_pub[i] + 2], s.n3);
  }
  s.d_kin = upload(kin, st);
  s.d_stick_of = upload(stick_of, st);
  s.d_zpos = upload(zpos, st);
  s.d_stick_off = upload(s.stick_off, st);
  s.d_stick_col = upload(s.stick_col, st);
  s.d_stick_y = upload(s.stick_y, st);
  s.d_col_x = upload(s.col_x, st);
  std::vector<int32_t> stick_at((size_t)s.ncols * s.n2, -1);
  for (int st_i = 0; st_i < s.nsticks; ++st_i)
    stick_at[(size_t)s.stick_col[st_i] * s.n2 + s.stick_y[st_i]] = st_i;
  std::vector<int16_t> xcol(s.n1, -1);
  for (int c = 0; c < s.ncols; ++c) xcol[s.col_x[c]] = (int16_t)c;
  s.d_stick_at = upload(stick_at, st);
  s.d_xcol = upload(xcol, st);
  std::vector<int32_t> shell_int(s.npw);
  for (int64_t i = 0; i < s.npw; ++i) shell_int[i] = s.shell_pub[s.int_to_pub[i]];
  s.d_shell = upload(shell_int, st);
  s.d_Tshell = upload(s.Tshell_h, st);
  // host vectors above die at scope end: wait for the copies
  PWH_CUDA(cudaStreamSynchronize(st));
}

// ------------------------------------------------------- device helpers -----
__global__ void k_potential_layout(const double* __restrict__ v, int n1, int n2, int n3,
                                   double scale, double* __restrict__ v64,
                                   float* __restrict__ v32, float2* __restrict__ vdf) {
  int64_t tot = (int64_t)n1 * n2 * n3;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    // t indexes the internal layout [i3][i2][i1]
    int i1 = (int)(t % n1);
    int64_t r = t / n1;
    int i2 = (int)(r % n2);
    int i3 = (int)(r / n2);
    double x = v[((int64_t)i1 * n2 + i2) * n3 + i3] * scale;
    v64[t] = x;
    v32[t] = (float)x;
    const float hi = __double2float_rn(x);
    vdf[t] = make_float2(hi, __double2float_rn(x - (double)hi));
  }
}

// sum of the (1/N^3-scaled) grid potential = mean V(r); one block, fixed order
__global__ void k_grid_sum(const double* __restrict__ v, int64_t n, double* __restrict__ out) {
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += v[i];
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out = t;
  }
}

__global__ void k_beta_gather(const double2* __restrict__ src, int64_t npw, int nproj,
                              const int32_t* __restrict__ int_to_pub,
                              double2* __restrict__ dst, float2* __restrict__ dst32) {
  int64_t tot = npw * nproj;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t % npw, p = t / npw;
    double2 z = src[p * npw + int_to_pub[i]];
    dst[t] = z;
    dst32[t] = make_float2((float)z.x, (float)z.y);
  }
}

void prepare_tc_projectors(System& s);  // tensor-core operand copies (gemm_tc.cu)

int* device_error_word(System& s) {
  if (!s.d_err) {
    PWH_CUDA(cudaMalloc((void**)&s.d_err, sizeof(int)));
    PWH_CUDA(cudaMemsetAsync(s.d_err, 0, sizeof(int), s.stream));
  }
  return s.d_err;
}

}  // namespace pwh

using namespace pwh;

extern "C" {

const char* pwh_last_error(void) { return g_last_error.c_str(); }

pwh_status pwh_create_system(const pwh_system_desc* desc, pwh_system** out) {
  return guarded([&] {
    PWH_CHECK_ARG(desc && out, "null argument");
    *out = nullptr;
    PWH_CHECK_ARG(std::isfinite(desc->ecut_ha) && desc->ecut_ha > 0, "ecut_ha must be > 0");
    PWH_CHECK_ARG(desc->precision >= PWH_FP64 && desc->precision <= PWH_MIXED_FAST,
                  "unknown precision");
    for (int d = 0; d < 3; ++d)
      PWH_CHECK_ARG(desc->fft[d] >= 0, "negative FFT size");
    for (int d = 0; d < 3; ++d)
      PWH_CHECK_ARG(std::isfinite(desc->kpoint[d]), "non-finite k-point");
    pwh_system* h = new pwh_system();
    System& s = h->s;
    try {
      std::memcpy(s.lattice, desc->lattice, sizeof(s.lattice));
      std::memcpy(s.kpoint, desc->kpoint, sizeof(s.kpoint));
      s.ecut = desc->ecut_ha;
      s.precision = desc->precision;
      s.stream = (cudaStream_t)desc->stream;
      build_basis(s, desc->fft);
      upload_basis(s);
      build_fft_plans(s);
      device_error_word(s);
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
  });
}

pwh_status pwh_destroy_system(pwh_system* sys) {
  return guarded([&] { delete sys; });
}

pwh_status pwh_get_dims(const pwh_system* sys, int64_t* npw, int32_t fft_out[3],
                        int64_t* nsticks) {
  return guarded([&] {
    PWH_CHECK_ARG(sys, "null system");
    if (npw) *npw = sys->s.npw;
    if (fft_out) {
      fft_out[0] = sys->s.n1; fft_out[1] = sys->s.n2; fft_out[2] = sys->s.n3;
    }
    if (nsticks) *nsticks = sys->s.nsticks;
  });
}

pwh_status pwh_get_miller(const pwh_system* sys, int32_t* miller) {
  return guarded([&] {
    PWH_CHECK_ARG(sys && miller, "null argument");
    std::memcpy(miller, sys->s.miller.data(), sys->s.miller.size() * sizeof(int32_t));
  });
}

pwh_status pwh_get_kinetic(const pwh_system* sys, double* kin) {
  return guarded([&] {
    PWH_CHECK_ARG(sys && kin, "null argument");
    std::memcpy(kin, sys->s.kin_pub.data(), sys->s.kin_pub.size() * sizeof(double));
  });
}

pwh_status pwh_get_internal_order(const pwh_system* sys, int32_t* int_to_pub) {
  return guarded([&] {
    PWH_CHECK_ARG(sys && int_to_pub, "null argument");
    std::memcpy(int_to_pub, sys->s.int_to_pub.data(), sys->s.int_to_pub.size() * sizeof(int32_t));
  });
}

pwh_status pwh_set_potential(pwh_system* sys, const double* v_r, int32_t on_device) {
  return guarded([&] {
    PWH_CHECK_ARG(sys && v_r, "null argument");
    System& s = sys->s;
    int64_t tot = (int64_t)s.n1 * s.n2 * s.n3;
    if (!s.d_v64) PWH_CUDA(cudaMalloc((void**)&s.d_v64, tot * sizeof(double)));
    if (!s.d_v32) PWH_CUDA(cudaMalloc((void**)&s.d_v32, tot * sizeof(float)));
    if (!s.d_vdf) PWH_CUDA(cudaMalloc((void**)&s.d_vdf, tot * sizeof(float2)));
    const double* src = v_r;
    double* tmp = nullptr;
    if (!on_device) {
      PWH_CUDA(cudaMalloc((void**)&tmp, tot * sizeof(double)));
      PWH_CUDA(cudaMemcpyAsync(tmp, v_r, tot * sizeof(double), cudaMemcpyHostToDevice, s.stream));
      src = tmp;
    }
    k_potential_layout<<<1024, 256, 0, s.stream>>>(src, s.n1, s.n2, s.n3, 1.0 / (double)tot,
                                                  s.d_v64, s.d_v32, s.d_vdf);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (tmp) {
      cudaStreamSynchronize(s.stream);
      cudaFree(tmp);
    }
    PWH_CUDA(e);
    double* dsum = nullptr;
    PWH_CUDA(cudaMalloc((void**)&dsum, sizeof(double)));
    k_grid_sum<<<1, 1024, 0, s.stream>>>(s.d_v64, tot, dsum);
    note_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&s.vbar, dsum, sizeof(double), cudaMemcpyDeviceToHost, s.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s.stream);
    cudaFree(dsum);
    PWH_CUDA(e);
    s.have_v = true;
  });
}

pwh_status pwh_set_projectors(pwh_system* sys, int32_t nproj, const void* beta,
                              const void* D, int32_t d_is_diag, int32_t on_device) {
  return guarded([&] {
    PWH_CHECK_ARG(sys, "null system");
    PWH_CHECK_ARG(nproj >= 0 && nproj <= 65536, "nproj out of range");
    System& s = sys->s;
    PWH_CUDA(cudaStreamSynchronize(s.stream));
    for (void** p : {(void**)&s.d_beta64, (void**)&s.d_ddiag, (void**)&s.d_dfull,
                     (void**)&s.d_beta32, (void**)&s.d_beta_bf16, (void**)&s.d_beta_bf16_t}) {
      if (*p) cudaFree(*p);
      *p = nullptr;
    }
    s.nproj = 0;
    s.gam_proj_ok = -1;
    // an overlap belongs to the projectors it was set with
    for (double2** p : {&s.d_q, &s.d_ksq}) {
      if (*p) cudaFree(*p);
      *p = nullptr;
    }
    s.have_overlap = false;
    if (nproj == 0) return;
    PWH_CHECK_ARG(beta && D, "null beta or D");
    size_t nb = (size_t)s.npw * nproj;
    PWH_CUDA(cudaMalloc((void**)&s.d_beta64, nb * sizeof(double2)));
    PWH_CUDA(cudaMalloc((void**)&s.d_beta32, nb * sizeof(float2)));
    const double2* src = (const double2*)beta;
    double2* tmp = nullptr;
    if (!on_device) {
      PWH_CUDA(cudaMalloc((void**)&tmp, nb * sizeof(double2)));
      PWH_CUDA(cudaMemcpyAsync(tmp, beta, nb * sizeof(double2), cudaMemcpyHostToDevice, s.stream));
      src = tmp;
    }
    k_beta_gather<<<2048, 256, 0, s.stream>>>(src, s.npw, nproj, s.d_int_to_pub, s.d_beta64,
                                             s.d_beta32);
    note_launch();
    cudaError_t e = cudaGetLastError();
    s.d_diag = d_is_diag != 0;
    size_t dn = s.d_diag ? (size_t)nproj * sizeof(double) : (size_t)nproj * nproj * sizeof(double2);
    void* ddst = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&ddst, dn);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ddst, D, dn, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          s.stream);
    if (s.d_diag) s.d_ddiag = (double*)ddst; else s.d_dfull = (double2*)ddst;
    cudaStreamSynchronize(s.stream);
    if (tmp) cudaFree(tmp);
    PWH_CUDA(e);
    s.nproj = nproj;
    prepare_tc_projectors(s);
  });
}

pwh_status pwh_set_precision(pwh_system* sys, int32_t precision) {
  return guarded([&] {
    PWH_CHECK_ARG(sys, "null system");
    PWH_CHECK_ARG(precision >= PWH_FP64 && precision <= PWH_MIXED_FAST, "unknown precision");
    sys->s.precision = precision;
  });
}

pwh_status pwh_set_kernel_timing(pwh_system* sys, int32_t on) {
  return guarded([&] {
    PWH_CHECK_ARG(sys, "null system");
    PWH_CUDA(cudaStreamSynchronize(sys->s.stream));
    sys->s.timer.reset();
    sys->s.timer.on = on != 0;
  });
}

pwh_status pwh_get_kernel_times(pwh_system* sys, pwh_kernel_time* out, int32_t max_out,
                                int32_t* count) {
  return guarded([&] {
    PWH_CHECK_ARG(sys && count && (out || max_out == 0), "null argument");
    PWH_CUDA(cudaStreamSynchronize(sys->s.stream));
    sys->s.timer.resolve();
    int c = 0;
    for (int f = 0; f < KF_COUNT; ++f) {
      if (c < max_out) {
        std::memset(out[c].name, 0, sizeof(out[c].name));
        std::strncpy(out[c].name, kKernelFamilyName[f], sizeof(out[c].name) - 1);
        out[c].launches = sys->s.timer.n[f];
        out[c].total_ms = sys->s.timer.ms[f];
        out[c].flops = sys->s.timer.flops[f];
        out[c].bytes = sys->s.timer.bytes[f];
      }
      ++c;
    }
    *count = c;
  });
}

pwh_status pwh_launch_count(int64_t* count) {
  return guarded([&] {
    PWH_CHECK_ARG(count, "null argument");
    *count = g_launches.load();
  });
}

pwh_status pwh_sync(pwh_system* sys) {
  return guarded([&] {
    PWH_CHECK_ARG(sys, "null system");
    System& s = sys->s;
    PWH_CUDA(cudaStreamSynchronize(s.stream));
    int e = 0;
    PWH_CUDA(cudaMemcpyAsync(&e, device_error_word(s), sizeof(int), cudaMemcpyDeviceToHost, s.stream));
    PWH_CUDA(cudaStreamSynchronize(s.stream));
    if (e != 0) {
      PWH_CUDA(cudaMemsetAsync(s.d_err, 0, sizeof(int), s.stream));
      throw Error{(pwh_status)e, "a bounded device wait gave up (kernel returned early)"};
    }
  });
}

}  // extern "C"
