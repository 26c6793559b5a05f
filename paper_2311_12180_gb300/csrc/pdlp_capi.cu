// C ABI of the GB300 PDLP solver (declared in include/pdlp.h): input
// validation, the sliced-ELL layout of K and K' (host, once per LP: the
// internal row order and the work items), the transpose of K, Sec. 2.2
// scaling and the sliced-ELL copies on the device, and the
// solve driver that replays a captured CUDA graph of one check period and
// polls a pinned copy of the device state one period behind, so the GPU never
// waits for the host.

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "pdlp.h"
#include "pdlp_host.h"
#include "pdlp_internal.cuh"
#include "pdlp_sell.h"
#include "pdlp_setup.cuh"

using namespace pdlp;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(PDLP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

constexpr int TRACE_CAP = 1 << 16;

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Layout {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  }
};

}  // namespace

int pdlp::set_error(int code, const char *msg) { return fail(code, msg ? msg : ""); }

struct pdlp_solver {
  int32_t m = 0, n = 0, n_eq = 0;
  int64_t nnz = 0;
  int device = 0;
  pdlp_params prm{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t cap_stream = nullptr;
  int num_sms = 0;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  SellMat K{}, KT{};
  char *sell_arena = nullptr;  // sliced-ELL copies of K and K', their work items
  size_t sell_bytes = 0;
  Vecs V{};
  DevState *st = nullptr;
  double *d_scal = nullptr;
  int32_t *K_ptr = nullptr, *K_idx = nullptr, *T_ptr = nullptr, *T_idx = nullptr;
  double *K_val = nullptr, *T_val = nullptr;
  double *D1 = nullptr, *D2 = nullptr, *work_m = nullptr, *work_n = nullptr;  // D1, D2: original order
  int32_t *perm_r = nullptr, *perm_c = nullptr;  // internal -> original row / column
  std::vector<int32_t> h_perm_r, h_perm_c;        // the same on the host (state export / import)
  pdlp_layout_info layout{};                      // sliced-ELL shapes of K and K'
  double *qd = nullptr;                           // QP: scaled Hessian diagonal (internal order), or null
  std::vector<double> h_qdiag;                    // QP: the caller's diagonal (state fingerprint)
  double *c = nullptr, *q = nullptr, *l = nullptr, *u = nullptr, *l0 = nullptr, *u0 = nullptr;
  int gridA = 1, gridB = 1, gridR1 = 1, gridR2 = 1, gridR3 = 1, gridI = 1;
  int slots = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  DevState *h_st = nullptr;    // pinned: state written by the host before a solve / read after
  DevState *h_poll = nullptr;  // pinned: two slots of polled state
  double *h_scal = nullptr;    // pinned
  double eta_hat0 = 1.0, omega0 = 1.0, q_norm = 0.0, c_norm = 0.0;
  double setup_ms = 0.0, solve_ms = 0.0, t0 = 0.0;
  int64_t launches = 0;
  int last_status = -1;
  bool have_result = false;
};

namespace {

// Dimensions, row starts and the vectors (host arrays).  The scans run in
// parallel chunks; the report names the first bad index of each kind.
int validate_vectors(int32_t m, int32_t n, int32_t n_eq, const double *c, const int32_t *rp, const double *q,
                     const double *l, const double *u) {
  if (m < 0 || n < 1 || n_eq < 0 || n_eq > m) return fail(PDLP_ERR_INVALID, "dimensions: need m >= 0, n >= 1, 0 <= n_eq <= m");
  if (!c || !rp || !l || !u || (m > 0 && !q)) return fail(PDLP_ERR_INVALID, "null input array");
  if (rp[0] != 0) return fail(PDLP_ERR_INVALID, "row_ptr[0] must be 0");
  const int T = host_threads((int64_t)m + n);
  std::vector<int32_t> bad_row(T, m), bad_c(T, n), bad_b(T, n), bad_q(T, m);
  parallel_for(T, [&](int t) {
    const int32_t i0 = (int32_t)((int64_t)m * t / T), i1 = (int32_t)((int64_t)m * (t + 1) / T);
    for (int32_t i = i0; i < i1; ++i)
      if (rp[i + 1] < rp[i]) {
        bad_row[t] = i;
        break;
      }
    for (int32_t i = i0; i < i1; ++i)
      if (!std::isfinite(q[i])) {
        bad_q[t] = i;
        break;
      }
    const int32_t j0 = (int32_t)((int64_t)n * t / T), j1 = (int32_t)((int64_t)n * (t + 1) / T);
    for (int32_t j = j0; j < j1; ++j)
      if (!std::isfinite(c[j])) {
        bad_c[t] = j;
        break;
      }
    for (int32_t j = j0; j < j1; ++j)
      if (std::isnan(l[j]) || std::isnan(u[j]) || l[j] > u[j] || l[j] == INFINITY || u[j] == -INFINITY) {
        bad_b[t] = j;
        break;
      }
  });
  const int32_t br = *std::min_element(bad_row.begin(), bad_row.end());
  if (br < m) return fail(PDLP_ERR_INVALID, "row_ptr is not non-decreasing at row " + std::to_string(br));
  const int32_t bc = *std::min_element(bad_c.begin(), bad_c.end()), bb = *std::min_element(bad_b.begin(), bad_b.end());
  if (bc < n && bc <= bb) return fail(PDLP_ERR_INVALID, "non-finite c at " + std::to_string(bc));
  if (bb < n) return fail(PDLP_ERR_INVALID, "bad bounds at variable " + std::to_string(bb));
  const int32_t bq = *std::min_element(bad_q.begin(), bad_q.end());
  if (bq < m) return fail(PDLP_ERR_INVALID, "non-finite q at row " + std::to_string(bq));
  return PDLP_OK;
}

int bad_entry(int64_t e, bool col_bad) {
  if (col_bad) return fail(PDLP_ERR_INVALID, "col_idx out of range at nonzero " + std::to_string(e));
  return fail(PDLP_ERR_INVALID, "non-finite matrix value at nonzero " + std::to_string(e));
}

// Column indices in [0, n) and finite values (host arrays); the report names
// the first bad nonzero.
int validate_entries(int64_t nnz, int32_t n, const int32_t *ci, const double *v) {
  if (nnz > 0 && (!ci || !v)) return fail(PDLP_ERR_INVALID, "null col_idx / val");
  // first bad nonzero, searched in parallel chunks
  const int T = host_threads(nnz);
  std::vector<int64_t> first(T, nnz);
  parallel_for(T, [&](int t) {
    for (int64_t e = nnz * t / T; e < nnz * (t + 1) / T; ++e)
      if (ci[e] < 0 || ci[e] >= n || !std::isfinite(v[e])) {
        first[t] = e;
        break;
      }
  });
  const int64_t e = *std::min_element(first.begin(), first.end());
  if (e < nnz) return bad_entry(e, ci[e] < 0 || ci[e] >= n);
  return PDLP_OK;
}

int check_params(const pdlp_params &p) {
  if (p.check_period < 1 || p.ruiz_iters < 0 || !(p.pc_alpha <= 2.0) || !(p.theta >= 0.0 && p.theta <= 1.0) ||
      !(p.eps_zero >= 0.0) || !(p.beta_suff > 0.0) || !(p.beta_nec > 0.0) || !(p.beta_art > 0.0) ||
      !(p.eps_infeas >= 0.0) ||
      (p.value_bits != 64 && p.value_bits != 32))
    return fail(PDLP_ERR_INVALID, "invalid parameters");
  return PDLP_OK;
}

void free_solver(pdlp_solver *s) {
  if (!s) return;
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  if (s->graph) cudaGraphDestroy(s->graph);
  for (auto &e : s->ev)
    if (e) cudaEventDestroy(e);
  if (s->arena) cudaFree(s->arena);
  if (s->sell_arena) cudaFree(s->sell_arena);
  if (s->qd) cudaFree(s->qd);
  if (s->h_st) cudaFreeHost(s->h_st);
  if (s->h_poll) cudaFreeHost(s->h_poll);
  if (s->h_scal) cudaFreeHost(s->h_scal);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

int build_graph(pdlp_solver *s) {
  if (s->gexec) return PDLP_OK;
  CK(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < s->slots && e == cudaSuccess; ++i) {
    e = launch_primal(s->KT, s->V, s->st, s->gridA, s->cap_stream);
    if (e == cudaSuccess) e = launch_dual(s->K, s->V, s->st, s->gridB, s->cap_stream);
  }
  if (e == cudaSuccess) e = launch_check_primal(s->KT, s->V, s->st, s->gridR1, s->cap_stream);
  if (e == cudaSuccess) e = launch_infeas(s->V, s->st, s->gridI, s->cap_stream);
  if (e == cudaSuccess) e = launch_check_dual(s->K, s->V, s->st, s->gridR2, s->cap_stream);
  if (e == cudaSuccess) e = launch_restart(s->V, s->st, s->gridR3, s->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s->cap_stream, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(PDLP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  if (e2 != cudaSuccess) return fail(PDLP_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e2));
  s->graph = g;
  CK(cudaGraphInstantiate(&s->gexec, s->graph, 0));
  return PDLP_OK;
}

int create_common(pdlp_solver **out, int32_t m, int32_t n, int32_t n_eq, const double *c, const int32_t *row_ptr,
                  const int32_t *col_idx, const double *val, const double *q, const double *l, const double *u,
                  const pdlp_params &prm, void *stream, bool dev_entries, double t_start);

}  // namespace

extern "C" {

void pdlp_default_params(pdlp_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->check_period = 64;
  p->ruiz_iters = 10;
  p->pc_alpha = 1.0;
  p->theta = 0.5;
  p->eps_zero = 1e-10;
  p->beta_suff = 0.2;
  p->beta_nec = 0.8;
  p->beta_art = 0.36;
  p->time_limit_s = 0.0;
  p->value_bits = 64;
  p->f32_polish = 1;
  p->eps_infeas = 1e-8;
}

const char *pdlp_last_error(void) { return g_err.c_str(); }

int pdlp_create_ex(pdlp_solver **out, int32_t m, int32_t n, int32_t n_eq, const double *c, const int32_t *row_ptr,
                   const int32_t *col_idx, const double *val, const double *q, const double *l, const double *u,
                   const pdlp_params *params, void *stream) {
  g_err.clear();
  if (!out) return fail(PDLP_ERR_INVALID, "out is NULL");
  pdlp_params prm;
  if (params)
    prm = *params;
  else
    pdlp_default_params(&prm);
  int rc = check_params(prm);
  if (rc) return rc;
  rc = validate_vectors(m, n, n_eq, c, row_ptr, q, l, u);
  if (rc) return rc;
  const double t_start = now_ms();
  const int64_t nnz = row_ptr[m];
  if (nnz >= ((int64_t)1 << 31)) return fail(PDLP_ERR_INVALID, "nnz must be < 2^31");
  rc = validate_entries(nnz, n, col_idx, val);
  if (rc) return rc;
  return create_common(out, m, n, n_eq, c, row_ptr, col_idx, val, q, l, u, prm, stream, false, t_start);
}

}  // extern "C"

namespace {

// The create path after validation.  c, row_ptr, q, l, u are host arrays;
// col_idx and val are host arrays, or device arrays when dev_entries.
int create_common(pdlp_solver **out, int32_t m, int32_t n, int32_t n_eq, const double *c, const int32_t *row_ptr,
                  const int32_t *col_idx, const double *val, const double *q, const double *l, const double *u,
                  const pdlp_params &prm, void *stream, bool dev_entries, double t_start) {
  const int64_t nnz = row_ptr[m];
  const cudaMemcpyKind entry_kind = dev_entries ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;

  // ---- host: the sliced-ELL layout of K (row lengths are known here) on a
  // host thread while the device takes the upload, builds K' and scales;
  // K''s layout comes from its row starts, on this thread while the device
  // scales ----
  SellLayout LK;
  struct Joiner {  // every exit waits for the layout thread
    std::thread t;
    ~Joiner() {
      if (t.joinable()) t.join();
    }
  } lk_thread;
  double qn = 0.0, cn = 0.0;  // ||q||^2, ||c||^2 of the original LP (Sec. 4.1), on the same thread
  lk_thread.t = std::thread([&LK, &qn, &cn, row_ptr, q, c, m, n, n_eq] {
    LK = sell_layout(row_ptr, m, n_eq);
    for (int32_t i = 0; i < m; ++i) qn += q[i] * q[i];
    for (int32_t j = 0; j < n; ++j) cn += c[j] * c[j];
  });

  pdlp_solver *s = new pdlp_solver();
  s->m = m;
  s->n = n;
  s->n_eq = n_eq;
  s->nnz = nnz;
  s->prm = prm;
#define CKS(call)                                                                                              \
  do {                                                                                                         \
    cudaError_t e_ = (call);                                                                                   \
    if (e_ != cudaSuccess) {                                                                                   \
      int code_ = (e_ == cudaErrorMemoryAllocation) ? PDLP_ERR_OOM : PDLP_ERR_CUDA;                          \
      std::string msg_ = std::string(#call) + ": " + cudaGetErrorString(e_);                                  \
      free_solver(s);                                                                                          \
      return fail(code_, msg_);                                                                                \
    }                                                                                                          \
  } while (0)
  CKS(cudaGetDevice(&s->device));
  int major = 0, minor = 0;
  CKS(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, s->device));
  CKS(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, s->device));
  CKS(cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device));
  CKS(kernels_init());
  if (stream) {
    s->stream = (cudaStream_t)stream;
  } else {
    CKS(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    s->own_stream = true;
  }
  CKS(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
  CKS(cudaEventCreateWithFlags(&s->ev[0], cudaEventDisableTiming));
  CKS(cudaEventCreateWithFlags(&s->ev[1], cudaEventDisableTiming));
  CKS(cudaMallocHost((void **)&s->h_st, sizeof(DevState)));
  CKS(cudaMallocHost((void **)&s->h_poll, 2 * sizeof(DevState)));
  CKS(cudaMallocHost((void **)&s->h_scal, 8 * sizeof(double)));
  std::memset(s->h_st, 0, sizeof(DevState));
  s->h_st->status = ST_RUNNING;

  // grids: the occupancy bound, at most one warp per work item (the K'
  // grids are set once its layout is known; the occupancy bound sizes the
  // partial-sum arrays)
  auto capped = [](int g, int nitems) {
    const int need = (nitems + NW - 1) / NW;
    return std::max(1, std::min(g, need));
  };
  const int gridA_max = occupancy_grid(KC_PRIMAL, s->num_sms), gridR1_max = occupancy_grid(KC_R1, s->num_sms);
  const int gridB_max = occupancy_grid(KC_DUAL, s->num_sms), gridR2_max = occupancy_grid(KC_R2, s->num_sms);
  s->gridA = gridA_max;
  s->gridB = gridB_max;  // capped by K's work items once its layout is known
  s->gridR1 = gridR1_max;
  s->gridR2 = gridR2_max;
  {
    const int64_t mx = n > m ? n : m;
    int g = occupancy_grid(KC_R3, s->num_sms);
    const int64_t need = (mx + NT - 1) / NT;
    s->gridR3 = (int)(need < g ? (need > 0 ? need : 1) : g);
    const int gi = occupancy_grid(KC_INFEAS, s->num_sms);
    s->gridI = (int)(need < gi ? (need > 0 ? need : 1) : gi);
  }
  const bool f32 = prm.value_bits == 32;

  // ---- one device arena for K, K' (CSR, original order: transpose and
  // scaling), the vectors and the state; a second one, once K''s layout is
  // known, for the sliced-ELL copies ----
  Layout L;
  const size_t M = (size_t)m, N = (size_t)n, Z = (size_t)nnz;
  const size_t o_Kptr = L.take(4 * (M + 1)), o_Kidx = L.take(4 * Z), o_Kval = L.take(8 * Z);
  const size_t o_Tptr = L.take(4 * (N + 1)), o_Tidx = L.take(4 * Z), o_Tval = L.take(8 * Z);
  const size_t nvec_n = 19, nvec_m = 15;
  const size_t o_vn = L.take(8 * N * nvec_n), o_vm = L.take(8 * (M + 1) * nvec_m);
  const size_t o_pr = L.take(4 * (M + 1)), o_pc = L.take(4 * N);
  const size_t o_pA = L.take(8 * (size_t)s->gridA * NV_A), o_pB = L.take(8 * (size_t)s->gridB * NV_B);
  const size_t o_pR1 = L.take(8 * (size_t)s->gridR1 * NV_R1), o_pR2 = L.take(8 * (size_t)s->gridR2 * NV_R2);
  const size_t o_pR3 = L.take(8 * (size_t)s->gridR3 * NV_R3), o_pI = L.take(8 * (size_t)s->gridI * NV_I);
  const size_t o_st = L.take(sizeof(DevState)), o_tr = L.take(sizeof(TraceRec) * TRACE_CAP);
  const size_t o_sc = L.take(8 * (8 + scalars_work_doubles()));
  const long long npw = 1LL << 20;  // exponent factors for the first 2^20 steps (16 MB)
  const size_t o_pw = L.take(16 * (size_t)npw);
  s->arena_bytes = L.off;
  CKS(cudaMalloc((void **)&s->arena, s->arena_bytes));
  char *A = s->arena;
  s->K_ptr = (int32_t *)(A + o_Kptr);
  s->K_idx = (int32_t *)(A + o_Kidx);
  s->K_val = (double *)(A + o_Kval);
  s->T_ptr = (int32_t *)(A + o_Tptr);
  s->T_idx = (int32_t *)(A + o_Tidx);
  s->T_val = (double *)(A + o_Tval);
  s->perm_r = (int32_t *)(A + o_pr);
  s->perm_c = (int32_t *)(A + o_pc);
  double *vn = (double *)(A + o_vn), *vm = (double *)(A + o_vm);
  auto VN = [&](int i) { return vn + (size_t)i * N; };
  auto VM = [&](int i) { return vm + (size_t)i * (M + 1); };
  // internal order: c~, l~, u~, D2, l, u (original bounds, for the output
  // projection), q~, D1; original order: D2, D1 (the scaling's result)
  s->c = VN(0);
  s->l = VN(1);
  s->u = VN(2);
  s->l0 = VN(4);
  s->u0 = VN(5);
  s->work_n = VN(16);
  s->D2 = VN(18);
  s->q = VM(0);
  s->work_m = VM(12);
  s->D1 = VM(14);
  s->st = (DevState *)(A + o_st);
  s->d_scal = (double *)(A + o_sc);

  Vecs &V = s->V;
  V.n = n;
  V.m = m;
  V.n_eq = n_eq;

  V.c = s->c;
  V.l = s->l;
  V.u = s->u;
  V.D2 = VN(3);
  V.l0 = s->l0;
  V.u0 = s->u0;
  V.q = s->q;
  V.D1 = VM(1);
  V.rD2 = VN(17);
  V.rD1 = VM(13);
  V.x[0] = VN(6);
  V.x[1] = VN(7);
  V.sx[0] = VN(8);
  V.sx[1] = VN(9);
  V.g = VN(10);
  V.gbar = VN(11);
  V.xlast = VN(12);
  V.xout = VN(13);
  V.g0 = VN(14);
  V.gprev = VN(15);
  V.kx0 = VM(11);
  V.gridI = s->gridI;
  V.y[0] = VM(2);
  V.y[1] = VM(3);
  V.sy[0] = VM(4);
  V.sy[1] = VM(5);
  V.Kx[0] = VM(6);
  V.Kx[1] = VM(7);
  V.Kxbar = VM(8);
  V.ylast = VM(9);
  V.yout = VM(10);
  V.partA = (double *)(A + o_pA);
  V.partB = (double *)(A + o_pB);
  V.partR1 = (double *)(A + o_pR1);
  V.partR2 = (double *)(A + o_pR2);
  V.partR3 = (double *)(A + o_pR3);
  V.partI = (double *)(A + o_pI);
  V.trace = (TraceRec *)(A + o_tr);
  V.pw = (const double *)(A + o_pw);
  V.npw = npw;
  V.perm_r = s->perm_r;
  V.perm_c = s->perm_c;

  // ---- transfers ----
  cudaStream_t st = s->stream;
  CKS(cudaMemsetAsync(s->arena, 0, s->arena_bytes, st));
  CKS(cudaMemcpyAsync(s->K_ptr, row_ptr, 4 * (M + 1), cudaMemcpyHostToDevice, st));
  if (nnz) {
    CKS(cudaMemcpyAsync(s->K_idx, col_idx, 4 * Z, entry_kind, st));
    CKS(cudaMemcpyAsync(s->K_val, val, 8 * Z, entry_kind, st));
  }

  // ---- K' on the device: row starts from K's column counts, then the
  // stable transpose (the threaded host counting sort when a column is
  // longer than the device's per-column sort takes) ----
  std::vector<int32_t> tp((size_t)n + 1, 0);
  int32_t longest = 0;
  // scratch of the row starts, then of the transpose; the transpose leaves
  // in it the permutation and entry rows that the scaling reuses (freed
  // after the scaling)
  const size_t wcs = col_starts_work_ints(n);
  struct ScratchBuffer {  // an error exit releases it (synchronously: the stream may be gone)
    void *p = nullptr;
    ~ScratchBuffer() {
      if (p) cudaFree(p);
    }
  } tw, lw;
  CKS(cudaMallocAsync(&tw.p, sizeof(int32_t) * (wcs + transpose_work_ints(n, nnz)), st));
  int32_t *const twork = static_cast<int32_t *>(tw.p);
  CKS(setup_col_starts(n, nnz, s->K_idx, s->T_ptr, twork, st));
  CKS(cudaMemcpyAsync(tp.data(), s->T_ptr, 4 * (N + 1), cudaMemcpyDeviceToHost, st));
  CKS(cudaMemcpyAsync(&longest, twork, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CKS(cudaStreamSynchronize(st));
  if (nnz && longest <= transpose_max_segment())
    CKS(setup_transpose(m, n, nnz, s->K_ptr, s->K_idx, s->K_val, s->T_ptr, s->T_idx, s->T_val, twork + wcs, st));
  const bool have_perm = nnz && longest <= transpose_max_segment();
  if (nnz && longest > transpose_max_segment()) {
    std::vector<int32_t> tp_h((size_t)n + 1), ti((size_t)nnz), ci_h;
    std::vector<double> tv((size_t)nnz), v_h;
    const int32_t *ci = col_idx;
    const double *v = val;
    if (dev_entries) {  // the host sort needs the entries on the host
      ci_h.resize(Z);
      v_h.resize(Z);
      CKS(cudaMemcpyAsync(ci_h.data(), s->K_idx, 4 * Z, cudaMemcpyDeviceToHost, st));
      CKS(cudaMemcpyAsync(v_h.data(), s->K_val, 8 * Z, cudaMemcpyDeviceToHost, st));
      CKS(cudaStreamSynchronize(st));
      ci = ci_h.data();
      v = v_h.data();
    }
    csr_transpose(m, n, row_ptr, ci, v, tp_h.data(), ti.data(), tv.data());
    CKS(cudaMemcpyAsync(s->T_idx, ti.data(), 4 * Z, cudaMemcpyHostToDevice, st));
    CKS(cudaMemcpyAsync(s->T_val, tv.data(), 8 * Z, cudaMemcpyHostToDevice, st));
    CKS(cudaStreamSynchronize(st));  // the host arrays go out of scope
  }
  // original c, q, l, u into spare vectors, consumed below
  CKS(cudaMemcpyAsync(V.xout, c, 8 * N, cudaMemcpyHostToDevice, st));
  if (m) CKS(cudaMemcpyAsync(V.yout, q, 8 * M, cudaMemcpyHostToDevice, st));
  double *const l_orig = VN(9), *const u_orig = VN(10);
  CKS(cudaMemcpyAsync(l_orig, l, 8 * N, cudaMemcpyHostToDevice, st));
  CKS(cudaMemcpyAsync(u_orig, u, 8 * N, cudaMemcpyHostToDevice, st));

  // ---- Sec. 2.2 scaling on the device (original order) ----
  {
    cudaError_t e;
    if (have_perm) {
      const int32_t *perm = twork + wcs + n, *rowid = perm + nnz;
      // reciprocal scratch: the x_last / y_last slots, unused until a solve begins
      e = setup_scale_perm(m, n, nnz, s->K_ptr, s->K_idx, s->K_val, s->T_ptr, s->T_val, rowid, perm, s->D1, s->D2,
                           s->work_m, s->work_n, VM(9), VN(12), prm.ruiz_iters, prm.pc_alpha, st);
    } else {
      e = setup_scale(m, n, nnz, s->K_ptr, s->K_idx, s->K_val, s->T_ptr, s->T_idx, s->T_val, s->D1, s->D2,
                      s->work_m, s->work_n, prm.ruiz_iters, prm.pc_alpha, st);
    }
    CKS(e);
    const cudaError_t ef = cudaFreeAsync(tw.p, st);
    tw.p = nullptr;
    CKS(ef);
  }
  // scaled vectors in the original order (spare slots), their scalars
  double *const c_s = VN(6), *const l_s = VN(7), *const u_s = VN(8), *const q_s = VM(2);
  CKS(setup_vectors(m, n, V.xout, V.yout, l_orig, u_orig, s->D1, s->D2, c_s, q_s, l_s, u_s, st));
  CKS(setup_scalars(m, n, nnz, c_s, q_s, s->K_val, s->d_scal, s->d_scal + 8, st));

  // the layout of K' (one group: every column of K) while the device scales
  SellLayout LT = sell_layout(tp.data(), n, n);
  lk_thread.t.join();
  s->q_norm = std::sqrt(qn);
  s->c_norm = std::sqrt(cn);
  s->gridB = capped(gridB_max, (int)LK.items.size());
  s->gridR2 = capped(gridR2_max, (int)LK.items.size());
  if (m) CKS(cudaMemcpyAsync(s->perm_r, LK.perm.data(), 4 * M, cudaMemcpyHostToDevice, st));
  if (LK.total >= ((int64_t)1 << 31) || LT.total >= ((int64_t)1 << 31)) {
    free_solver(s);
    return fail(PDLP_ERR_INVALID, "the sliced-ELL copy of K needs 2^31 or more stored entries");
  }
  s->gridA = capped(gridA_max, (int)LT.items.size());
  s->gridR1 = capped(gridR1_max, (int)LT.items.size());
  V.gridA = s->gridA;
  V.gridR1 = s->gridR1;
  CKS(cudaMemcpyAsync(s->perm_c, LT.perm.data(), 4 * N, cudaMemcpyHostToDevice, st));
  // ---- sliced-ELL copies of the scaled K and K', columns renumbered ----
  {
    Layout SL;
    const size_t ZK = (size_t)LK.total, ZT = (size_t)LT.total;
    const size_t o_ki = SL.take(4 * ZK), o_kv = SL.take(8 * ZK), o_kf = f32 ? SL.take(4 * ZK) : 0;
    const size_t o_ti = SL.take(4 * ZT), o_tv = SL.take(8 * ZT), o_tf = f32 ? SL.take(4 * ZT) : 0;
    const size_t o_kit = SL.take(sizeof(int4) * LK.items.size()), o_tit = SL.take(sizeof(int4) * LT.items.size());
    s->sell_bytes = SL.off;
    CKS(cudaMalloc((void **)&s->sell_arena, s->sell_bytes));
    char *B = s->sell_arena;
    s->K = SellMat{m, (int32_t)LK.items.size(), (const int4 *)(B + o_kit), (const int32_t *)(B + o_ki),
                   (const double *)(B + o_kv), f32 ? (const float *)(B + o_kf) : nullptr};
    s->KT = SellMat{n, (int32_t)LT.items.size(), (const int4 *)(B + o_tit), (const int32_t *)(B + o_ti),
                    (const double *)(B + o_tv), f32 ? (const float *)(B + o_tf) : nullptr};
    // the solve's CUDA graph (one check period) is captured and instantiated
    // now, on the host, while the device is still scaling: it needs only the
    // pointers and grids, all known here
    s->slots = prm.check_period + (prm.check_period / 8 > 4 ? prm.check_period / 8 : 4);
    {
      const int grc = build_graph(s);
      if (grc) {
        free_solver(s);
        return grc;
      }
    }
    if (!LK.items.empty())
      CKS(cudaMemcpyAsync(B + o_kit, LK.items.data(), sizeof(int4) * LK.items.size(), cudaMemcpyHostToDevice, st));
    CKS(cudaMemcpyAsync(B + o_tit, LT.items.data(), sizeof(int4) * LT.items.size(), cudaMemcpyHostToDevice, st));
    // scratch: inverse permutations, entry bases and strides of both layouts
    Layout WL;
    const size_t o_ir = WL.take(4 * (M + 1)), o_ic = WL.take(4 * N), o_bk = WL.take(4 * (M + 1)),
                 o_bt = WL.take(4 * N), o_lk = WL.take(M + 1), o_lt = WL.take(N);
    CKS(cudaMallocAsync(&lw.p, WL.off, st));
    char *W = static_cast<char *>(lw.p);
    int32_t *inv_r = (int32_t *)(W + o_ir), *inv_c = (int32_t *)(W + o_ic);
    if (m) {
      CKS(cudaMemcpyAsync(W + o_bk, LK.base.data(), 4 * M, cudaMemcpyHostToDevice, st));
      CKS(cudaMemcpyAsync(W + o_lk, LK.lane.data(), M, cudaMemcpyHostToDevice, st));
    }
    CKS(cudaMemcpyAsync(W + o_bt, LT.base.data(), 4 * N, cudaMemcpyHostToDevice, st));
    CKS(cudaMemcpyAsync(W + o_lt, LT.lane.data(), N, cudaMemcpyHostToDevice, st));
    CKS(setup_invert(m, s->perm_r, inv_r, st));
    CKS(setup_invert(n, s->perm_c, inv_c, st));
    CKS(setup_sell_fill(m, LK.total, s->perm_r, (const int32_t *)(W + o_bk), (const uint8_t *)(W + o_lk), s->K_ptr,
                        s->K_idx, s->K_val, inv_c, (int32_t *)s->K.idx, (double *)s->K.val, st));
    CKS(setup_sell_fill(n, LT.total, s->perm_c, (const int32_t *)(W + o_bt), (const uint8_t *)(W + o_lt), s->T_ptr,
                        s->T_idx, s->T_val, inv_r, (int32_t *)s->KT.idx, (double *)s->KT.val, st));
    if (f32) {
      CKS(setup_f32(LK.total, s->K.val, (float *)s->K.val32, st));
      CKS(setup_f32(LT.total, s->KT.val, (float *)s->KT.val32, st));
    }
    // debug mode (environment PDLP_DEBUG_CHECKS=1): every index the step and
    // check kernels will gather through, and every work item they will walk,
    // is checked on the device before the first solve
    const char *dbg = std::getenv("PDLP_DEBUG_CHECKS");
    if (dbg && dbg[0] == '1') {
      unsigned int ck[3], ct[3];
      CKS(setup_check_sell(m, n, LK.total, (int32_t)LK.items.size(), (const int4 *)(B + o_kit), s->K.idx, s->K.val,
                           s->K.val32, ck, st));
      CKS(setup_check_sell(n, m, LT.total, (int32_t)LT.items.size(), (const int4 *)(B + o_tit), s->KT.idx,
                           s->KT.val, s->KT.val32, ct, st));
      if (ck[0] | ck[1] | ck[2] | ct[0] | ct[1] | ct[2]) {
        free_solver(s);
        return fail(PDLP_ERR_INVALID, "debug check of the sliced-ELL copies failed: K entries / items / rows " +
                                          std::to_string(ck[0]) + " / " + std::to_string(ck[1]) + " / " +
                                          std::to_string(ck[2]) + ", K' " + std::to_string(ct[0]) + " / " +
                                          std::to_string(ct[1]) + " / " + std::to_string(ct[2]));
      }
    }
    // the host layouts go out of scope: wait for their uploads
    CKS(cudaStreamSynchronize(st));
    const cudaError_t ef = cudaFreeAsync(lw.p, st);
    lw.p = nullptr;
    CKS(ef);
  }
  s->layout.K_stored = LK.total;
  s->layout.K_slices = LK.nslices;
  s->layout.K_long_rows = LK.nlong;
  s->layout.KT_stored = LT.total;
  s->layout.KT_slices = LT.nslices;
  s->layout.KT_long_rows = LT.nlong;
  s->layout.long_threshold = SELL_LONG;
  s->h_perm_r.swap(LK.perm);
  s->h_perm_c.swap(LT.perm);
  // ---- vectors in the internal order ----
  CKS(setup_permute(n, s->perm_c, c_s, s->c, st));
  CKS(setup_permute(n, s->perm_c, l_s, s->l, st));
  CKS(setup_permute(n, s->perm_c, u_s, s->u, st));
  CKS(setup_permute(n, s->perm_c, s->D2, VN(3), st));
  CKS(setup_permute(n, s->perm_c, l_orig, s->l0, st));
  CKS(setup_permute(n, s->perm_c, u_orig, s->u0, st));
  CKS(setup_permute(m, s->perm_r, q_s, s->q, st));
  CKS(setup_permute(m, s->perm_r, s->D1, VM(1), st));
  CKS(setup_recip(n, VN(3), VN(17), st));
  CKS(setup_recip(m, VM(1), VM(13), st));
  CKS(setup_pow_table((double *)(A + o_pw), npw, st));
  CKS(cudaMemcpyAsync(s->h_scal, s->d_scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CKS(cudaStreamSynchronize(st));
  const double cc = std::sqrt(s->h_scal[0]), qq = std::sqrt(s->h_scal[1]), kmax = s->h_scal[2];
  s->eta_hat0 = kmax > 0.0 ? 1.0 / kmax : 1.0;                                        // Algorithm 1
  s->omega0 = (cc > prm.eps_zero && qq > prm.eps_zero) ? cc / qq : 1.0;              // InitializePrimalWeight
  s->setup_ms = now_ms() - t_start;
#undef CKS
  *out = s;
  return PDLP_OK;
}

}  // namespace

extern "C" {

int pdlp_create_device(pdlp_solver **out, int32_t m, int32_t n, int32_t n_eq, const double *c,
                       const int32_t *row_ptr, const int32_t *col_idx, const double *val, const double *q,
                       const double *l, const double *u, const pdlp_params *params, void *stream) {
  g_err.clear();
  if (!out) return fail(PDLP_ERR_INVALID, "out is NULL");
  pdlp_params prm;
  if (params)
    prm = *params;
  else
    pdlp_default_params(&prm);
  int rc = check_params(prm);
  if (rc) return rc;
  if (m < 0 || n < 1 || n_eq < 0 || n_eq > m) return fail(PDLP_ERR_INVALID, "dimensions: need m >= 0, n >= 1, 0 <= n_eq <= m");
  if (!c || !row_ptr || !l || !u || (m > 0 && !q)) return fail(PDLP_ERR_INVALID, "null input array");
  const double t_start = now_ms();
  cudaStream_t st = (cudaStream_t)stream;
  // the row starts and the vectors come to the host (the layout and the
  // checks need them; the norms are taken by the same host code as in
  // pdlp_create_ex); the entries stay on the device
  std::vector<int32_t> rp((size_t)m + 1);
  std::vector<double> hc((size_t)n), hl((size_t)n), hu((size_t)n), hq((size_t)m);
  CK(cudaMemcpyAsync(rp.data(), row_ptr, 4 * ((size_t)m + 1), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hc.data(), c, 8 * (size_t)n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hl.data(), l, 8 * (size_t)n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hu.data(), u, 8 * (size_t)n, cudaMemcpyDeviceToHost, st));
  if (m) CK(cudaMemcpyAsync(hq.data(), q, 8 * (size_t)m, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  rc = validate_vectors(m, n, n_eq, hc.data(), rp.data(), hq.data(), hl.data(), hu.data());
  if (rc) return rc;
  const int64_t nnz = rp[m];
  if (nnz >= ((int64_t)1 << 31)) return fail(PDLP_ERR_INVALID, "nnz must be < 2^31");
  if (nnz > 0) {
    if (!col_idx || !val) return fail(PDLP_ERR_INVALID, "null col_idx / val");
    int64_t first = nnz;
    int col_bad = 0;
    CK(setup_check_entries(nnz, col_idx, val, n, &first, &col_bad, st));
    if (first < nnz) return bad_entry(first, col_bad != 0);
  }
  return create_common(out, m, n, n_eq, hc.data(), rp.data(), col_idx, val, hq.data(), hl.data(), hu.data(), prm,
                       stream, true, t_start);
}

int pdlp_create(pdlp_solver **out, int32_t m, int32_t n, int32_t n_eq, const double *c, const int32_t *row_ptr,
                const int32_t *col_idx, const double *val, const double *q, const double *l, const double *u) {
  return pdlp_create_ex(out, m, n, n_eq, c, row_ptr, col_idx, val, q, l, u, nullptr, nullptr);
}

void pdlp_destroy(pdlp_solver *s) {
  if (!s) return;
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  free_solver(s);
}

int pdlp_begin(pdlp_solver *s, const double *x0, const double *y0, double tol, int64_t max_iter) {
  g_err.clear();
  if (!s) return fail(PDLP_ERR_INVALID, "solver is NULL");
  if (!(tol >= 0.0) || max_iter < 1) return fail(PDLP_ERR_INVALID, "need tol >= 0 and max_iter >= 1");
  CK(cudaSetDevice(s->device));
  int rc = build_graph(s);
  if (rc) return rc;
  cudaStream_t st = s->stream;
  Vecs &V = s->V;
  const size_t N = (size_t)s->n, M = (size_t)s->m;
  if (x0) CK(cudaMemcpyAsync(V.xout, x0, 8 * N, cudaMemcpyHostToDevice, st));
  if (y0 && M) CK(cudaMemcpyAsync(V.yout, y0, 8 * M, cudaMemcpyHostToDevice, st));
  CK(setup_warm_perm(s->m, s->n, x0 ? V.xout : nullptr, (y0 && M) ? V.yout : nullptr, s->perm_r, s->perm_c, V.D1,
                     V.D2, V.x[0], V.y[0], st));
  CK(cudaMemsetAsync(V.sx[0], 0, 8 * N, st));
  CK(cudaMemsetAsync(V.sx[1], 0, 8 * N, st));
  CK(cudaMemcpyAsync(V.xlast, V.x[0], 8 * N, cudaMemcpyDeviceToDevice, st));
  if (M) {
    CK(cudaMemsetAsync(V.sy[0], 0, 8 * M, st));
    CK(cudaMemsetAsync(V.sy[1], 0, 8 * M, st));
    CK(cudaMemcpyAsync(V.ylast, V.y[0], 8 * M, cudaMemcpyDeviceToDevice, st));
  }
  CK(cudaStreamSynchronize(st));  // h_st may still be read by an earlier async copy
  DevState &h = *s->h_st;
  std::memset(&h, 0, sizeof(DevState));
  h.eta = s->eta_hat0;
  h.omega = s->omega0;
  h.W = 0.0;
  h.tol = tol;
  h.q_norm = s->q_norm;
  h.c_norm = s->c_norm;
  h.theta = s->prm.theta;
  h.eps_zero = s->prm.eps_zero;
  h.beta_suff = s->prm.beta_suff;
  h.beta_nec = s->prm.beta_nec;
  h.beta_art = s->prm.beta_art;
  h.rel_kkt_best = INFINITY;
  h.max_iter = max_iter;
  h.f64_switch_k = -1;
  h.cur = 0;
  h.need_g = 1;
  h.check_pending = 1;
  h.status = ST_RUNNING;
  h.mode = MODE_INIT;
  h.P = s->prm.check_period;
  h.trace_cap = TRACE_CAP;
  h.use_f32 = s->prm.value_bits == 32 ? 1 : 0;
  h.polish = s->prm.f32_polish ? 1 : 0;
  h.eps_infeas = s->V.qd ? 0.0 : s->prm.eps_infeas;  // the certificates are the LP's
  CK(cudaMemcpyAsync(s->st, s->h_st, sizeof(DevState), cudaMemcpyHostToDevice, st));
  // KKT(z^{0,0}): K'y, Kx and the pieces of eq. (kkt) at the start point
  CK(launch_check_primal(s->KT, V, s->st, s->gridR1, st));
  CK(launch_check_dual(s->K, V, s->st, s->gridR2, st));
  s->launches = 0;
  s->have_result = false;
  s->last_status = ST_RUNNING;
  s->t0 = now_ms();
  return PDLP_OK;
}

int pdlp_run_periods(pdlp_solver *s, int32_t n_periods) {
  g_err.clear();
  if (!s || !s->gexec) return fail(PDLP_ERR_INVALID, "call pdlp_begin first");
  CK(cudaSetDevice(s->device));
  for (int32_t i = 0; i < n_periods; ++i) {
    CK(cudaGraphLaunch(s->gexec, s->stream));
    s->launches++;
  }
  return PDLP_OK;
}

int pdlp_poll(pdlp_solver *s, int *status, int64_t *iters) {
  g_err.clear();
  if (!s) return fail(PDLP_ERR_INVALID, "solver is NULL");
  CK(cudaSetDevice(s->device));
  CK(cudaMemcpyAsync(&s->h_poll[0], s->st, sizeof(DevState), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (status) *status = s->h_poll[0].status;
  if (iters) *iters = s->h_poll[0].k;
  return PDLP_OK;
}

int pdlp_finish(pdlp_solver *s, double *x_out, double *y_out, int *status, int64_t *iters) {
  g_err.clear();
  if (!s) return fail(PDLP_ERR_INVALID, "solver is NULL");
  CK(cudaSetDevice(s->device));
  cudaStream_t st = s->stream;
  CK(launch_output(s->V, s->st, st));
  CK(cudaMemcpyAsync(s->h_st, s->st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
  if (x_out) CK(cudaMemcpyAsync(x_out, s->V.xout, 8 * (size_t)s->n, cudaMemcpyDeviceToHost, st));
  if (y_out && s->m) CK(cudaMemcpyAsync(y_out, s->V.yout, 8 * (size_t)s->m, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  s->solve_ms = now_ms() - s->t0;
  s->have_result = true;
  s->last_status = s->h_st->status;
  if (status) *status = s->h_st->status;
  if (iters) *iters = s->h_st->k;
  return PDLP_OK;
}

// Replays the graph until the device state leaves RUNNING (or the time
// limit), polling a pinned copy of the state one period behind, then writes
// the outputs (pdlp_finish).
static int drive(pdlp_solver *s, double *x_out, double *y_out, int *status, int64_t *iters) {
  cudaStream_t st = s->stream;
  const double limit_ms = s->prm.time_limit_s > 0.0 ? 1000.0 * s->prm.time_limit_s : INFINITY;
  // one period in flight ahead of the one being polled
  int slot = 0;
  CK(cudaGraphLaunch(s->gexec, st));
  s->launches++;
  CK(cudaMemcpyAsync(&s->h_poll[slot], s->st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
  CK(cudaEventRecord(s->ev[slot], st));
  for (;;) {
    const int nxt = slot ^ 1;
    CK(cudaGraphLaunch(s->gexec, st));
    s->launches++;
    CK(cudaMemcpyAsync(&s->h_poll[nxt], s->st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(s->ev[nxt], st));
    CK(cudaEventSynchronize(s->ev[slot]));
    if (s->h_poll[slot].status != ST_RUNNING) break;
    if (now_ms() - s->t0 > limit_ms) {
      CK(launch_time_limit(s->st, st));
      break;
    }
    slot = nxt;
  }
  return pdlp_finish(s, x_out, y_out, status, iters);
}

int pdlp_solve_warm(pdlp_solver *s, const double *x0, const double *y0, double tol, int64_t max_iter, double *x_out,
                    double *y_out, int *status, int64_t *iters) {
  int rc = pdlp_begin(s, x0, y0, tol, max_iter);
  if (rc) return rc;
  return drive(s, x_out, y_out, status, iters);
}

int pdlp_resume(pdlp_solver *s, double *x_out, double *y_out, int *status, int64_t *iters) {
  g_err.clear();
  if (!s || !s->gexec) return fail(PDLP_ERR_INVALID, "pdlp_resume: call pdlp_begin or pdlp_set_state first");
  CK(cudaSetDevice(s->device));
  CK(cudaStreamSynchronize(s->stream));
  CK(cudaMemcpy(s->h_st, s->st, sizeof(DevState), cudaMemcpyDeviceToHost));
  if (s->h_st->status != ST_RUNNING) return pdlp_finish(s, x_out, y_out, status, iters);
  return drive(s, x_out, y_out, status, iters);
}

int pdlp_solve(pdlp_solver *s, double tol, int64_t max_iter, double *x_out, double *y_out, int *status,
               int64_t *iters) {
  return pdlp_solve_warm(s, nullptr, nullptr, tol, max_iter, x_out, y_out, status, iters);
}

int32_t pdlp_kernel_count(void) { return KC_NUM; }
const char *pdlp_kernel_name(int32_t i) { return kernel_class_name(i); }

int pdlp_time_kernels(pdlp_solver *s, int32_t n_periods, double *ms, int64_t *launches) {
  g_err.clear();
  if (!s || !ms || !launches) return fail(PDLP_ERR_INVALID, "null argument");
  CK(cudaSetDevice(s->device));
  cudaStream_t st = s->stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto timed = [&](int kc, cudaError_t (*fn)(pdlp_solver *, cudaStream_t)) -> int {
    CK(cudaEventRecord(e0, st));
    CK(fn(s, st));
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, e0, e1));
    ms[kc] += t;
    launches[kc] += 1;
    return PDLP_OK;
  };
  auto poll = [&](DevState &out) -> int {
    CK(cudaMemcpyAsync(&s->h_poll[0], s->st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out = s->h_poll[0];
    return PDLP_OK;
  };
  int rc = PDLP_OK;
  int done = 0;
  DevState h;
  while (done < n_periods && rc == PDLP_OK) {
    if ((rc = poll(h))) break;
    if (h.status != ST_RUNNING) break;
    if (!h.check_pending) {
      rc = timed(h.need_g ? KC_PRIMAL : KC_PRIMAL_REUSE,
                 [](pdlp_solver *t, cudaStream_t q) { return launch_primal(t->KT, t->V, t->st, t->gridA, q); });
      if (!rc) rc = timed(KC_DUAL, [](pdlp_solver *t, cudaStream_t q) { return launch_dual(t->K, t->V, t->st, t->gridB, q); });
      continue;
    }
    rc = timed(KC_R1, [](pdlp_solver *t, cudaStream_t q) { return launch_check_primal(t->KT, t->V, t->st, t->gridR1, q); });
    if (!rc && h.mode == MODE_CHECK && h.eps_infeas > 0.0)
      rc = timed(KC_INFEAS, [](pdlp_solver *t, cudaStream_t q) { return launch_infeas(t->V, t->st, t->gridI, q); });
    if (!rc) rc = timed(KC_R2, [](pdlp_solver *t, cudaStream_t q) { return launch_check_dual(t->K, t->V, t->st, t->gridR2, q); });
    if (!rc) rc = poll(h);
    if (!rc && h.status == ST_RUNNING && h.restart_to)
      rc = timed(KC_R3, [](pdlp_solver *t, cudaStream_t q) { return launch_restart(t->V, t->st, t->gridR3, q); });
    ++done;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

int pdlp_get_info(const pdlp_solver *s, pdlp_info *info) {
  g_err.clear();
  if (!s || !info) return fail(PDLP_ERR_INVALID, "null argument");
  const DevState &h = *s->h_st;
  std::memset(info, 0, sizeof(*info));
  info->status = s->have_result ? h.status : -1;
  info->which = h.which;
  info->iters = h.k;
  info->attempts = h.attempts;
  info->restarts = h.restarts;
  info->checks = h.checks;
  info->pobj = h.term[0];
  info->dobj = h.term[1];
  info->rp_norm = h.term[2];
  info->rd_norm = h.term[3];
  info->q_norm = s->q_norm;
  info->c_norm = s->c_norm;
  info->omega = h.omega;
  info->eta_hat = h.eta;
  info->setup_ms = s->setup_ms;
  info->solve_ms = s->solve_ms;
  info->graph_launches = s->launches;
  info->f64_switch_iter = h.f64_switch_k;
  if (info->status == ST_PRIMAL_INFEASIBLE || info->status == ST_DUAL_INFEASIBLE) {
    info->ray_obj = h.ray[0];
    info->ray_res = h.ray[1];
  }
  return PDLP_OK;
}

int pdlp_get_trace(const pdlp_solver *s, pdlp_check *trace, int32_t cap, int32_t *count) {
  g_err.clear();
  if (!s || (cap > 0 && !trace)) return fail(PDLP_ERR_INVALID, "null argument");
  CK(cudaSetDevice(s->device));
  const int nt = s->h_st->ntrace;
  if (count) *count = nt;
  // retained: the last TRACE_CAP records, the oldest at index first % TRACE_CAP
  const int kept = nt < TRACE_CAP ? nt : TRACE_CAP, first = nt - kept;
  const int ncopy = kept < cap ? kept : cap;
  if (ncopy <= 0) return PDLP_OK;
  std::vector<TraceRec> tmp(kept);
  CK(cudaMemcpy(tmp.data(), s->V.trace, sizeof(TraceRec) * kept, cudaMemcpyDeviceToHost));
  for (int i = 0; i < ncopy; ++i) {
    const TraceRec &r = tmp[(first + i) % TRACE_CAP];
    trace[i].k = r.k;
    trace[i].attempts = r.attempts;
    trace[i].restarts = r.restarts;
    trace[i].restart = r.restart;
    trace[i].cand_avg = r.cand_avg;
    trace[i].kkt_cur = r.kkt_cur;
    trace[i].kkt_avg = r.kkt_avg;
    trace[i].kkt_start = r.kkt_start;
    trace[i].omega = r.omega;
    trace[i].eta_hat = r.eta_hat;
    trace[i].rel_gap = r.rel_gap;
    trace[i].rel_primal = r.rel_primal;
    trace[i].rel_dual = r.rel_dual;
  }
  return PDLP_OK;
}

int pdlp_get_scaling(const pdlp_solver *s, double *D1, double *D2, double *val_scaled) {
  g_err.clear();
  if (!s) return fail(PDLP_ERR_INVALID, "solver is NULL");
  CK(cudaSetDevice(s->device));
  CK(cudaStreamSynchronize(s->stream));
  if (D1 && s->m) CK(cudaMemcpy(D1, s->D1, 8 * (size_t)s->m, cudaMemcpyDeviceToHost));
  if (D2) CK(cudaMemcpy(D2, s->D2, 8 * (size_t)s->n, cudaMemcpyDeviceToHost));
  if (val_scaled && s->nnz) CK(cudaMemcpy(val_scaled, s->K_val, 8 * (size_t)s->nnz, cudaMemcpyDeviceToHost));
  return PDLP_OK;
}

// ---- solver state (checkpoint / resume) ----
//
// Blob: StateHeader, the DevState bytes, then the scaled-space vectors in the
// ORIGINAL order of rows and columns (exact: a permutation moves bits, it
// rounds nothing): n-vectors x, sum eta x, K'y, x at the last restart, K'y at
// the epoch start, K'y of the previous accepted iterate; m-vectors y,
// sum eta y, Kx, y at the last restart, Kx at the epoch start.  Together with
// the LP and the parameters these fix every later step (Algorithm 1's
// z^{n,t}, the epoch sums behind z-bar, eta, omega, k, t, n, the KKT
// references and the restart candidate); the other buffers are rewritten
// before they are read again.
namespace {
struct StateHeader {
  uint64_t magic;
  uint32_t version;
  int32_t m, n, check_period, value_bits, pad;
  int64_t nnz;
  uint64_t devstate_bytes;
  uint64_t fingerprint;  // of the LP as the solver holds it (see lp_fingerprint)
};
constexpr uint64_t STATE_MAGIC = 0x3154535050444c50ull;  // "PLDPPST1" little-endian
constexpr int STATE_NV_N = 6, STATE_NV_M = 5;

// FNV-1a over the internal row and column orders and the norms and start
// scalars derived from c, q and the scaled K: two LPs that differ in these
// cannot exchange states.
uint64_t lp_fingerprint(const pdlp_solver *s) {
  uint64_t h = 0xcbf29ce484222325ull;
  auto mix = [&h](const void *p, size_t bytes) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < bytes; ++i) h = (h ^ b[i]) * 0x100000001b3ull;
  };
  mix(s->h_perm_r.data(), 4 * s->h_perm_r.size());
  mix(s->h_perm_c.data(), 4 * s->h_perm_c.size());
  const double sc[4] = {s->q_norm, s->c_norm, s->eta_hat0, s->omega0};
  mix(sc, sizeof(sc));
  mix(&s->n_eq, sizeof(s->n_eq));
  mix(s->h_qdiag.data(), 8 * s->h_qdiag.size());
  return h;
}

size_t state_bytes(const pdlp_solver *s) {
  return sizeof(StateHeader) + sizeof(DevState) + 8 * ((size_t)STATE_NV_N * s->n + (size_t)STATE_NV_M * s->m);
}

void state_vectors(const pdlp_solver *s, int cur, double *(&vn)[STATE_NV_N], double *(&vm)[STATE_NV_M]) {
  const Vecs &V = s->V;
  double *const n_vecs[STATE_NV_N] = {V.x[cur], V.sx[cur], V.g, V.xlast, V.g0, V.gprev};
  double *const m_vecs[STATE_NV_M] = {V.y[cur], V.sy[cur], V.Kx[cur], V.ylast, V.kx0};
  for (int i = 0; i < STATE_NV_N; ++i) vn[i] = n_vecs[i];
  for (int i = 0; i < STATE_NV_M; ++i) vm[i] = m_vecs[i];
}
}  // namespace

int pdlp_get_state(const pdlp_solver *s, void *buf, size_t cap, size_t *bytes) {
  g_err.clear();
  if (!s) return fail(PDLP_ERR_INVALID, "solver is NULL");
  const size_t need = state_bytes(s);
  if (bytes) *bytes = need;
  if (!buf) return PDLP_OK;
  if (cap < need) return fail(PDLP_ERR_INVALID, "pdlp_get_state: buffer smaller than the state");
  CK(cudaSetDevice(s->device));
  CK(cudaStreamSynchronize(s->stream));
  char *out = static_cast<char *>(buf);
  StateHeader h{};
  h.magic = STATE_MAGIC;
  h.version = 1;
  h.m = s->m;
  h.n = s->n;
  h.check_period = s->prm.check_period;
  h.value_bits = s->prm.value_bits;
  h.nnz = s->nnz;
  h.devstate_bytes = sizeof(DevState);
  h.fingerprint = lp_fingerprint(s);
  std::memcpy(out, &h, sizeof(h));
  DevState d;
  CK(cudaMemcpy(&d, s->st, sizeof(DevState), cudaMemcpyDeviceToHost));
  d.ntrace = 0;  // the check trace stays with the solver that recorded it
  std::memcpy(out + sizeof(h), &d, sizeof(d));
  double *vn[STATE_NV_N], *vm[STATE_NV_M];
  state_vectors(s, d.cur, vn, vm);
  double *dst = reinterpret_cast<double *>(out + sizeof(h) + sizeof(d));
  std::vector<double> tmp((size_t)std::max(s->n, s->m));
  auto pull = [&](const double *src, int32_t count, const std::vector<int32_t> &perm) -> int {
    if (count == 0) return PDLP_OK;
    CK(cudaMemcpy(tmp.data(), src, 8 * (size_t)count, cudaMemcpyDeviceToHost));
    for (int32_t r = 0; r < count; ++r) dst[perm[r]] = tmp[r];
    dst += count;
    return PDLP_OK;
  };
  for (int i = 0; i < STATE_NV_N; ++i)
    if (int rc = pull(vn[i], s->n, s->h_perm_c)) return rc;
  for (int i = 0; i < STATE_NV_M; ++i)
    if (int rc = pull(vm[i], s->m, s->h_perm_r)) return rc;
  return PDLP_OK;
}

int pdlp_set_state(pdlp_solver *s, const void *buf, size_t bytes) {
  g_err.clear();
  if (!s || !buf) return fail(PDLP_ERR_INVALID, "null argument");
  if (bytes != state_bytes(s)) return fail(PDLP_ERR_INVALID, "pdlp_set_state: size does not match this solver's state");
  const char *in = static_cast<const char *>(buf);
  StateHeader h;
  std::memcpy(&h, in, sizeof(h));
  if (h.magic != STATE_MAGIC || h.version != 1 || h.devstate_bytes != sizeof(DevState))
    return fail(PDLP_ERR_INVALID, "pdlp_set_state: not a state of this library version");
  if (h.m != s->m || h.n != s->n || h.nnz != s->nnz || h.check_period != s->prm.check_period ||
      h.value_bits != s->prm.value_bits || h.fingerprint != lp_fingerprint(s))
    return fail(PDLP_ERR_INVALID, "pdlp_set_state: the state belongs to another LP or other parameters");
  DevState d;
  std::memcpy(&d, in + sizeof(h), sizeof(d));
  if ((d.cur != 0 && d.cur != 1) || d.check_pending != 0)
    return fail(PDLP_ERR_INVALID, "pdlp_set_state: the state was not taken between check periods");
  // the fields the kernels index or divide with: the check period, the
  // trace ring (its size and write position), the step count (the exponent
  // table), and the FP32 values, which exist only with value_bits = 32
  if (d.P != s->prm.check_period || d.trace_cap != TRACE_CAP || d.ntrace != 0 || d.k < 0 || d.t < 0 ||
      d.attempts < d.k || d.max_iter < 1 || (d.use_f32 != 0 && d.use_f32 != 1) ||
      (d.use_f32 && s->prm.value_bits != 32) || (d.need_g != 0 && d.need_g != 1))
    return fail(PDLP_ERR_INVALID, "pdlp_set_state: the state's counters or flags are out of range");
  CK(cudaSetDevice(s->device));
  int rc = build_graph(s);
  if (rc) return rc;
  double *vn[STATE_NV_N], *vm[STATE_NV_M];
  state_vectors(s, d.cur, vn, vm);
  const double *src = reinterpret_cast<const double *>(in + sizeof(h) + sizeof(d));
  std::vector<double> tmp((size_t)std::max(s->n, s->m));
  cudaStream_t st = s->stream;
  CK(cudaStreamSynchronize(st));
  auto push = [&](double *dst, int32_t count, const std::vector<int32_t> &perm) -> int {
    if (count == 0) return PDLP_OK;
    for (int32_t r = 0; r < count; ++r) tmp[r] = src[perm[r]];
    CK(cudaMemcpy(dst, tmp.data(), 8 * (size_t)count, cudaMemcpyHostToDevice));
    src += count;
    return PDLP_OK;
  };
  for (int i = 0; i < STATE_NV_N; ++i)
    if ((rc = push(vn[i], s->n, s->h_perm_c))) return rc;
  for (int i = 0; i < STATE_NV_M; ++i)
    if ((rc = push(vm[i], s->m, s->h_perm_r))) return rc;
  std::memset(d.cnt, 0, sizeof(d.cnt));
  *s->h_st = d;
  CK(cudaMemcpy(s->st, s->h_st, sizeof(DevState), cudaMemcpyHostToDevice));
  s->launches = 0;
  s->have_result = false;
  s->last_status = d.status;
  s->t0 = now_ms();
  return PDLP_OK;
}

int pdlp_set_quadratic(pdlp_solver *s, const double *qdiag) {
  g_err.clear();
  if (!s) return fail(PDLP_ERR_INVALID, "solver is NULL");
  if (qdiag)
    for (int32_t j = 0; j < s->n; ++j)
      if (!std::isfinite(qdiag[j]) || qdiag[j] < 0.0)
        return fail(PDLP_ERR_INVALID, "pdlp_set_quadratic: need finite, non-negative diagonal entries (variable " +
                                          std::to_string(j) + ")");
  CK(cudaSetDevice(s->device));
  CK(cudaStreamSynchronize(s->stream));
  // the captured graph holds the kernels' arguments: rebuilt at the next begin
  if (s->gexec) {
    cudaGraphExecDestroy(s->gexec);
    s->gexec = nullptr;
  }
  if (s->graph) {
    cudaGraphDestroy(s->graph);
    s->graph = nullptr;
  }
  if (!qdiag) {
    s->V.qd = nullptr;
    s->h_qdiag.clear();
    return PDLP_OK;
  }
  s->h_qdiag.assign(qdiag, qdiag + s->n);
  if (!s->qd) CK(cudaMalloc((void **)&s->qd, 8 * (size_t)s->n));
  CK(cudaMemcpyAsync(s->V.xout, qdiag, 8 * (size_t)s->n, cudaMemcpyHostToDevice, s->stream));
  CK(setup_qp_diag(s->n, s->perm_c, s->V.D2, s->V.xout, s->qd, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  s->V.qd = s->qd;
  return PDLP_OK;
}

int pdlp_get_layout(const pdlp_solver *s, pdlp_layout_info *info) {
  g_err.clear();
  if (!s || !info) return fail(PDLP_ERR_INVALID, "null argument");
  *info = s->layout;
  return PDLP_OK;
}

void *pdlp_get_stream(const pdlp_solver *s) { return s ? (void *)s->stream : nullptr; }

size_t pdlp_device_bytes(const pdlp_solver *s) { return s ? s->arena_bytes + s->sell_bytes : 0; }

}  // extern "C"
