// Host side of the PDDSparse assembly library: geometry of Sec. 3.1
// (knots, patches, extended stencils, CSR pattern), device tables, TMA
// descriptors, launch configuration and the C ABI of pdds.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "pdds.h"
#include "pdds_internal.h"

namespace pdds {
// Dynamic shared memory of the tcgen05 network kernel ahead of its unit ring,
// and its launch with the network's FP32 vectors (host, 5 x 64: W1[:, 0],
// W1[:, 1], b1, b2, w3) as a kernel parameter (pdds_path_net.cu).
size_t net_smem_bytes();
cudaError_t launch_path_kernel_net(int coef, bool rec, bool ext, const KParams& kp,
                                   const float* w, int grid, int block, size_t smem,
                                   cudaStream_t stream);
}  // namespace pdds

using pdds::KnotDesc;
using pdds::ProbDesc;

namespace {

thread_local std::string g_last_error = "no error";

// ------------------------------------------------------------ geometry
// Knots live on the lattice (i, j), 0 <= i <= LX = Hx m, 0 <= j <= LY = Hy m;
// a lattice point is an unknown knot when it is interior and lies on a grid
// line (i % m == 0 or j % m == 0).  Knots are numbered row by row (j), then
// by i, which gives the closed-form index below.
struct Geometry {
  pdds_grid g{};
  int LX = 0, LY = 0;
  double dx = 0, dy = 0;
  int64_t n = 0, nnz = 0;
  std::vector<int32_t> ki, kj, row_ptr, col, slot2csr;
  std::vector<KnotDesc> kd;
  int max_slots = 0;

  bool is_knot(int i, int j) const {
    if (i <= 0 || i >= LX || j <= 0 || j >= LY) return false;
    return (i % g.m == 0) || (j % g.m == 0);
  }
  int64_t index(int i, int j) const {
    const int64_t full = (j - 1) / g.m;      // grid-line rows below j
    const int64_t part = (j - 1) - full;     // other rows below j
    const int64_t before = full * (LX - 1) + part * (int64_t)(g.Hx - 1);
    const int64_t pos = (j % g.m == 0) ? (i - 1) : (i / g.m - 1);
    return before + pos;
  }
};

bool build_geometry(const pdds_grid& g, Geometry& G, bool with_tables, std::string& err) {
  if (!(g.x1 > g.x0) || !(g.y1 > g.y0) || !std::isfinite(g.x0) || !std::isfinite(g.x1) ||
      !std::isfinite(g.y0) || !std::isfinite(g.y1)) {
    err = "grid: need x1 > x0 and y1 > y0 (finite)";
    return false;
  }
  if (g.Hx < 1 || g.Hy < 1 || g.m < 1 || g.ext < 0 || (g.Hx < 2 && g.Hy < 2)) {
    err = "grid: need Hx, Hy >= 1 with one of them >= 2, m >= 1, ext >= 0";
    return false;
  }
  if ((int64_t)g.Hx * g.m > (1 << 20) || (int64_t)g.Hy * g.m > (1 << 20)) {
    err = "grid: Hx*m and Hy*m must be <= 2^20";
    return false;
  }
  G.g = g;
  G.LX = g.Hx * g.m;
  G.LY = g.Hy * g.m;
  G.dx = (g.x1 - g.x0) / G.LX;
  G.dy = (g.y1 - g.y0) / G.LY;
  G.n = (int64_t)(g.Hy - 1) * (G.LX - 1) + (int64_t)(G.LY - 1 - (g.Hy - 1)) * (g.Hx - 1);
  if (G.n <= 0 || G.n > (int64_t)1 << 30) {
    err = "grid: knot count out of range";
    return false;
  }
  G.ki.resize(G.n);
  G.kj.resize(G.n);
  {
    int64_t k = 0;
    for (int j = 1; j < G.LY; ++j) {
      if (j % g.m == 0)
        for (int i = 1; i < G.LX; ++i) { G.ki[k] = i; G.kj[k] = j; ++k; }
      else
        for (int i = g.m; i < G.LX; i += g.m) { G.ki[k] = i; G.kj[k] = j; ++k; }
    }
    if (k != G.n) { err = "internal: knot enumeration mismatch"; return false; }
  }
  G.row_ptr.assign(G.n + 1, 0);
  if (with_tables) G.kd.resize(G.n);
  std::vector<int64_t> cols;
  // Two passes: sizes, then contents.
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      G.nnz = G.row_ptr[G.n];
      G.col.resize(G.nnz);
    }
    int64_t slots_total = 0;
    for (int64_t k = 0; k < G.n; ++k) {
      const int i = G.ki[k], j = G.kj[k], m = g.m, E = g.ext;
      // slab (Eq. 13) = patch (Eq. 15): Omega is a grid-aligned rectangle
      int ilo, ihi, jlo, jhi;
      if (i % m == 0) { ilo = i - m; ihi = i + m; } else { ilo = (i / m) * m; ihi = ilo + m; }
      if (j % m == 0) { jlo = j - m; jhi = j + m; } else { jlo = (j / m) * m; jhi = jlo + m; }
      const int line[4] = {ihi, jhi, ilo, jlo};
      const int lo_along[4] = {jlo, ilo, jlo, ilo};
      const int hi_along[4] = {jhi, ihi, jhi, ihi};
      const int lmax_along[4] = {G.LY, G.LX, G.LY, G.LX};
      const int lmax_line[4] = {G.LX, G.LY, G.LX, G.LY};
      cols.clear();
      cols.push_back(k);
      KnotDesc d{};
      int nslots = 0;
      for (int o = 0; o < 4; ++o) {
        const bool dir = (line[o] == 0 || line[o] == lmax_line[o]);
        const int a = std::max(lo_along[o] - E, 0);
        const int b = std::min(hi_along[o] + E, lmax_along[o]);
        d.line[o] = line[o];
        d.a[o] = a;
        d.b[o] = b;
        if (dir) {
          d.dirbits |= 1 << o;
          d.off[o] = -1;
          continue;
        }
        d.off[o] = nslots;
        nslots += b - a + 1;
        const bool vertical = (o == 0 || o == 2);
        for (int t = a; t <= b; ++t) {
          const int pi = vertical ? line[o] : t, pj = vertical ? t : line[o];
          if (G.is_knot(pi, pj)) cols.push_back(G.index(pi, pj));
        }
      }
      std::sort(cols.begin(), cols.end());
      cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
      if (pass == 0) {
        G.row_ptr[k + 1] = G.row_ptr[k] + (int32_t)cols.size();
        if ((int64_t)G.row_ptr[k + 1] > (int64_t)INT32_MAX / 2) {
          err = "grid: nnz exceeds int32 range";
          return false;
        }
        continue;
      }
      std::copy(cols.begin(), cols.end(), G.col.begin() + G.row_ptr[k]);
      G.max_slots = std::max(G.max_slots, nslots);
      if (!with_tables) continue;
      d.xk = (float)(g.x0 + i * G.dx);
      d.yk = (float)(g.y0 + j * G.dy);
      d.box[0] = (float)((ilo - i) * G.dx);
      d.box[1] = (float)((ihi - i) * G.dx);
      d.box[2] = (float)((jlo - j) * G.dy);
      d.box[3] = (float)((jhi - j) * G.dy);
      d.ki = i;
      d.kj = j;
      d.slot_base = (int32_t)slots_total;
      d.nslots = nslots;
      G.kd[k] = d;
      for (int o = 0; o < 4; ++o) {
        if (d.off[o] < 0) continue;
        const bool vertical = (o == 0 || o == 2);
        for (int t = d.a[o]; t <= d.b[o]; ++t) {
          const int pi = vertical ? line[o] : t, pj = vertical ? t : line[o];
          int32_t csr = -1;
          if (G.is_knot(pi, pj)) {
            const int64_t c = G.index(pi, pj);
            const auto it = std::lower_bound(cols.begin(), cols.end(), c);
            csr = G.row_ptr[k] + (int32_t)(it - cols.begin());
          }
          G.slot2csr.push_back(csr);
        }
      }
      slots_total += nslots;
    }
  }
  return true;
}

// ---------------------------------------------------------- TMA encode
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
size_t round_up(size_t a, size_t b) { return (a + b - 1) / b * b; }

}  // namespace

// ================================================================ context
struct pdds_ctx {
  pdds_grid grid{};
  int coef_id = 0;
  double params[8] = {0};
  int tab_nx = 0, tab_ny = 0;
  Geometry geo;
  double s_min = 0, s_max = 0;  // diffusion bounds (step-cap rule)
  int device = 0, num_sms = 0;
  // device tables
  KnotDesc* d_knots = nullptr;
  int32_t* d_slot2csr = nullptr;
  int32_t* d_row_ptr = nullptr;
  int32_t* d_col = nullptr;
  float* d_tab = nullptr;  // sigma then c, padded rows
  CUtensorMap* d_tmap = nullptr;
  int tile_w = 0, tile_h = 0;
  pdds::Scratch* d_scratch = nullptr;
  int64_t* d_unit_prefix = nullptr;
  int64_t* d_path_prefix = nullptr;
  int64_t* d_prob_prefix = nullptr;
  // launch configuration
  int block = 256, ctas_per_sm = 0, exit_batch = 4;
  int64_t unit_paths = 4096;
  int64_t k_max = 0;
  uint32_t tag = 0;  // Philox tag (fourth counter word) of single-problem calls
  int net_engine = PDDS_NET_TCGEN05;  // tensor-core engine of the in-path network
  float net_w[5 * 64] = {};  // the attached network's W1[:, 0], W1[:, 1], b1, b2, w3
  int batch_calls = 0;  // > 0: Philox calls between exit checks of a batched launch
  bool timing = false;
  bool timing_pending = false;  // ev0/ev1 recorded around a path kernel, time not read yet
  double wait_s = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // solver scratch
  double* d_work = nullptr;
  pdds::SolveScalars* d_scalars = nullptr;
  // end-to-end scratch
  int64_t* e_N = nullptr;
  int32_t* e_rp = nullptr;
  int32_t* e_col = nullptr;
  double *e_val = nullptr, *e_b = nullptr, *e_u = nullptr;
  // batch launch cache
  ProbDesc* d_batch = nullptr;
  int batch_cap = 0;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cap_stream = nullptr;
  // control variate (staged network image) and whether it is on
  void* d_mlp = nullptr;
  int cv_mode = 0;               // 0 none, 1 in-path network, 2 tabulated gradient
  float* d_cvtab = nullptr;      // [cv_ny-1][cv_nx-1][8] cell corners of grad u0 (mode 2), owned
  int cv_nx = 0, cv_ny = 0;
  double dom_bound_all = 0.0;  // set by a batched launch: max |coordinate| of all its domains
  // exit scheme and per-knot steps (extended-exit kernels)
  int scheme = PDDS_SCHEME_EM;
  double* d_hknot = nullptr;  // owned copy of h_k, or nullptr
  double h_min = 0;           // smallest h_k (wait bound)
  // stencil interpolation: linear, or RBF with device tables
  std::vector<int> stencil_len[2];  // distinct interface-stencil lengths per orientation
  int interp = PDDS_INTERP_LINEAR;
  double rbf_shape = 0;
  float* d_rbf_coef = nullptr;
  int64_t* d_rbf_off = nullptr;
  int rbf_deg = 0, rbf_lmax = 0;
  // calibration scratch: records of the naive and the GM pass, a CSR and b
  pdds_path_record* cal_rec = nullptr;
  int64_t cal_rec_cap = 0;    // records per pass
  double *cal_val = nullptr, *cal_b = nullptr;
  int32_t *cal_rp = nullptr, *cal_col = nullptr;
  std::vector<uint64_t> graph_key;
  pdds_stats_t st{};
  std::string err = "no error";
};

namespace {

pdds_status fail(pdds_ctx* c, pdds_status s, const std::string& msg) {
  if (c) c->err = msg; else g_last_error = msg;
  return s;
}
pdds_status cuda_fail(pdds_ctx* c, cudaError_t e, const char* what) {
  return fail(c, PDDS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define CK(ctx, call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

// The path-kernel time of the last timed assembly: waits for its end event
// only here, so that timing adds no host synchronization to the assembly.
pdds_status read_timing(pdds_ctx* c) {
  if (!c->timing_pending) return PDDS_OK;
  c->timing_pending = false;
  CK(c, cudaEventSynchronize(c->ev1));
  CK(c, cudaEventElapsedTime(&c->st.path_kernel_ms, c->ev0, c->ev1));
  return PDDS_OK;
}

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
}

void free_ctx(pdds_ctx* c) {
  if (!c) return;
  cudaFree(c->d_knots); cudaFree(c->d_slot2csr); cudaFree(c->d_row_ptr); cudaFree(c->d_col);
  cudaFree(c->d_tab); cudaFree(c->d_tmap); cudaFree(c->d_scratch); cudaFree(c->d_unit_prefix);
  cudaFree(c->d_path_prefix); cudaFree(c->d_prob_prefix); cudaFree(c->d_work);
  cudaFree(c->d_scalars); cudaFree(c->e_N); cudaFree(c->e_rp); cudaFree(c->e_col);
  cudaFree(c->e_val); cudaFree(c->e_b); cudaFree(c->e_u); cudaFree(c->d_batch);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  cudaFree(c->d_mlp);
  cudaFree(c->d_hknot); cudaFree(c->cal_rec); cudaFree(c->cal_val); cudaFree(c->cal_b);
  cudaFree(c->cal_rp); cudaFree(c->cal_col);
  cudaFree(c->d_rbf_coef); cudaFree(c->d_rbf_off); cudaFree(c->d_cvtab);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  delete c;
}

// Bounds of s(x) for the default step cap.
void sigma_bounds(const pdds_coeffs& cf, const std::vector<float>& sig, double& lo, double& hi) {
  const double r2 = std::sqrt(2.0);
  switch (cf.builtin_id) {
    case PDDS_COEF_VARSIGMA: lo = 0.7 * r2; hi = 1.3 * r2; break;
    case PDDS_COEF_TABLE:
      lo = 1e300; hi = 0;
      for (float v : sig) { lo = std::min(lo, (double)v); hi = std::max(hi, (double)v); }
      break;
    case PDDS_COEF_CONSTANT: lo = hi = std::fabs(cf.params[0]); break;
    default: lo = hi = r2;
  }
}

size_t stage_bytes(const pdds_ctx* c) {
  size_t b = pdds::stage_header_bytes() + round_up((size_t)c->geo.max_slots * 8, 128);
  if (c->coef_id == PDDS_COEF_TABLE) b += round_up((size_t)2 * c->tile_w * c->tile_h * 4, 128);
  return round_up(b, 128);
}

ProbDesc make_prob(const pdds_ctx* c, int tag) {
  ProbDesc D{};
  const Geometry& G = c->geo;
  D.coef_id = c->coef_id;
  D.n = (int32_t)G.n;
  D.LX = G.LX;
  D.LY = G.LY;
  for (int i = 0; i < 8; ++i) D.params[i] = (float)c->params[i];
  D.x0 = (float)c->grid.x0; D.y0 = (float)c->grid.y0;
  D.x1 = (float)c->grid.x1; D.y1 = (float)c->grid.y1;
  D.dx = (float)G.dx; D.dy = (float)G.dy;
  D.inv_dx = (float)(1.0 / G.dx); D.inv_dy = (float)(1.0 / G.dy);
  if (c->coef_id == PDDS_COEF_TABLE) {
    D.tab_inv_dx = (float)((c->tab_nx - 1) / (c->grid.x1 - c->grid.x0));
    D.tab_inv_dy = (float)((c->tab_ny - 1) / (c->grid.y1 - c->grid.y0));
    D.tmap = c->d_tmap;
    D.tab_nx = c->tab_nx;
    D.tab_ny = c->tab_ny;
  }
  D.tag = tag;
  D.sigma_max = (float)(c->s_max * (1.0 + 1e-6));  // bilinear lookups may round up 1 ulp
  D.h_per_knot = c->d_hknot;
  if (c->cv_mode == 2) {
    D.cv_tab = c->d_cvtab;
    D.cv_nx = c->cv_nx;
    D.cv_ny = c->cv_ny;
    D.cv_inv_dx = (float)((c->cv_nx - 1) / (c->grid.x1 - c->grid.x0));
    D.cv_inv_dy = (float)((c->cv_ny - 1) / (c->grid.y1 - c->grid.y0));
  }
  if (c->interp == PDDS_INTERP_RBF) {
    D.rbf_coef = c->d_rbf_coef;
    D.rbf_off = c->d_rbf_off;
    D.rbf_deg = c->rbf_deg;
    D.rbf_lmax = c->rbf_lmax;
  }
  D.knots = c->d_knots;
  D.slot2csr = c->d_slot2csr;
  D.col = c->d_col;
  return D;
}

pdds_status check_csr(pdds_ctx* c, const pdds_csr* G, const double* b) {
  if (!G || !b || !G->row_ptr || !G->col || !G->val)
    return fail(c, PDDS_EINVAL, "assemble: G (row_ptr, col, val) and b must be device pointers");
  if (G->n != c->geo.n || G->nnz != c->geo.nnz)
    return fail(c, PDDS_EINVAL, "assemble: G sized differently from pdds_num_knots");
  return PDDS_OK;
}

// Order of a path's step count: a quarter of the smaller subdomain side
// squared over s_max^2 h (about the mean exit time of a patch from its knot,
// in steps: 195 for config 2, 7.6 for config 5, 120-1500 for config 3).
double mean_steps_estimate(const pdds_ctx* c, double dt) {
  const double Lx = (c->grid.x1 - c->grid.x0) / c->grid.Hx;
  const double Ly = (c->grid.y1 - c->grid.y0) / c->grid.Hy;
  const double L = std::min(Lx, Ly);
  return 0.25 * L * L / (std::max(c->s_max * c->s_max, 1e-300) * dt);
}
// Philox calls (two steps each) a warp takes between its exit checks: one
// sixteenth of the expected steps per path, within [2, 8] -- longer runs
// between checks save the warp's ballots and branches (measured on one GB300:
// 8 calls instead of 2 is 3.2 % faster on config 3 and 3.4 % on config 2, and
// 1.2 % slower on config 5's ~11-step paths, which keep 2).
int calls_per_check(const pdds_ctx* c, double dt) {
  const double k = mean_steps_estimate(c, dt) / 16.0;
  return (int)std::min(8.0, std::max(2.0, std::round(k)));
}

int64_t default_kmax(const pdds_ctx* c, double dt) {
  const double Lx = (c->grid.x1 - c->grid.x0) / c->grid.Hx;
  const double Ly = (c->grid.y1 - c->grid.y0) / c->grid.Hy;
  const double T = std::pow(std::min(Lx, Ly), 2) / std::pow(std::max(c->s_min, 1e-12), 2);
  return (int64_t)std::ceil(40.0 * T / dt);
}

// Everything one or more problems need for one persistent launch.
// ext: extended-exit kernel (per-knot steps and/or the Gobet-Menozzi shift gm).
pdds_status run_paths(pdds_ctx* c, const ProbDesc& p0, const ProbDesc* d_probs, int nprob,
                      double dt, uint64_t seed, int64_t kmax, pdds::PathRecordDev* rec,
                      cudaStream_t stream, size_t sbytes, int max_slots, int tile_w, int tile_h,
                      int coef_id, bool ext = false, bool gm = false,
                      pdds::PathRecordDev* rec_gm = nullptr) {
  pdds::KParams kp{};
  kp.prob0 = p0;
  kp.probs = d_probs;
  kp.nprob = nprob;
  kp.prob_unit_prefix = c->d_prob_prefix;
  kp.exit_batch = c->exit_batch;
  kp.calls_per_check = c->batch_calls > 0 ? c->batch_calls : calls_per_check(c, dt);
  kp.unit_paths = c->unit_paths;
  kp.scratch = c->d_scratch;
  kp.records = rec;
  kp.key0 = (uint32_t)seed;
  kp.key1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {  // Philox4x32-10 key schedule (Weyl constants)
    kp.round_keys[2 * r] = kp.key0 + (uint32_t)r * 0x9E3779B9u;
    kp.round_keys[2 * r + 1] = kp.key1 + (uint32_t)r * 0xBB67AE85u;
  }
  kp.h = (float)dt;
  kp.sqh = (float)std::sqrt(dt);
  kp.kmax = kmax;
  kp.dt = dt;
  kp.gm = gm ? 1 : 0;
  kp.max_slots = max_slots;
  kp.tile_w = tile_w;
  kp.tile_h = tile_h;
  kp.stage_bytes = (int)sbytes;
  kp.mixed = rec_gm != nullptr ? 1 : 0;
  kp.records_gm = rec_gm;
  // a wait may outlast the slowest path of a unit: K_max steps at ~4 us
  // (per-knot steps: the longest cap is kmax dt / h_min steps)
  const double kmax_eff = ext && c->d_hknot && c->h_min < dt ? (double)kmax * dt / c->h_min
                                                             : (double)kmax;
  kp.wait_ns = c->wait_s > 0 ? (uint64_t)(c->wait_s * 1e9) : (uint64_t)(10e9 + 4000.0 * kmax_eff);
  // cv 3: the in-path network on tcgen05 (the warpgroup kernel)
  int cv = nprob == 1 ? c->cv_mode : 0;
  if (cv == 1 && c->net_engine == PDDS_NET_TCGEN05) cv = 3;
  kp.mlp = cv == 1 || cv == 3 ? c->d_mlp : nullptr;
  {
    // the largest |coordinate| of the launch's domains (problem 0 here, the
    // batch caller gives the bound over all of them) decides whether the
    // coefficient set's angles may skip the reduction
    const pdds_grid& g = c->grid;
    const double b0 = std::max(std::max(std::fabs(g.x0), std::fabs(g.x1)),
                               std::max(std::fabs(g.y0), std::fabs(g.y1)));
    const double B = nprob == 1 ? b0 : c->dom_bound_all;
    const double lim = coef_id == PDDS_COEF_POISSON_E1 ? 256.0
                       : coef_id == PDDS_COEF_VARSIGMA   ? 7.0
                                                          : 1.0;
    kp.trig_direct = B <= lim ? 1 : 0;
  }
  // the network step is ~10x heavier: wait bounds scale with it
  if ((cv == 1 || cv == 3) && c->wait_s <= 0) kp.wait_ns = (uint64_t)(10e9 + 40000.0 * kmax_eff);
  // network kernels keep the staged network at the start of dynamic shared
  // memory (the tcgen05 kernel: its swizzled operand tiles)
  const size_t smem = 2 * sbytes + (cv == 1   ? round_up(pdds::mlp_image_bytes(), 128)
                                    : cv == 3 ? pdds::net_smem_bytes()
                                              : 0);
  CK(c, pdds::set_path_kernel_smem(coef_id, rec != nullptr, cv, ext, smem));
  // network: <= 256 threads; the tcgen05 kernel takes one warpgroup
  const int block = cv == 1 ? std::min(c->block, 256) : cv == 3 ? 128 : c->block;
  int per_sm = c->ctas_per_sm;
  if (per_sm <= 0) {
    CK(c, pdds::path_kernel_occupancy(coef_id, rec != nullptr, cv, ext, block, smem, &per_sm));
    if (per_sm <= 0) return fail(c, PDDS_EINVAL, "launch: block/shared memory too large");
  }
  // tcgen05 kernel: 96 TMEM columns per CTA, 512 per SM
  if (cv == 3) per_sm = std::min(per_sm, 512 / 96);
  const int grid = c->num_sms * per_sm;
  c->st.path_grid = grid;
  c->st.path_block = block;
  if (c->timing) CK(c, cudaEventRecord(c->ev0, stream));
  if (cv == 3)
    CK(c, pdds::launch_path_kernel_net(coef_id, rec != nullptr, ext, kp, c->net_w, grid, block,
                                       smem, stream));
  else
    CK(c, pdds::launch_path_kernel(coef_id, rec != nullptr, cv, ext, kp, grid, block, smem, stream));
  if (c->timing) CK(c, cudaEventRecord(c->ev1, stream));
  return PDDS_OK;
}

// scheme: PDDS_SCHEME_EM / _GM, or -1 for the context's setting.  rec_gm
// (with rec, GM scheme): the mixed GM/EM run, Gobet-Menozzi exits to rec_gm,
// naive exits to rec and into G and b.
pdds_status assemble_impl(pdds_ctx* c, const int64_t* N, int64_t Nu, double dt, uint64_t seed,
                          pdds_csr* G, double* b, pdds_path_record* rec, cudaStream_t s,
                          int scheme = -1, pdds_path_record* rec_gm = nullptr) {
  (void)cudaGetLastError();  // a failed call elsewhere must not be reported here
  if (!(dt > 0) || !std::isfinite(dt)) return fail(c, PDDS_EINVAL, "assemble: dt must be > 0");
  if (!N && (Nu < 1 || Nu >= ((int64_t)1 << 31)))
    return fail(c, PDDS_EINVAL, "assemble: n_paths must be in [1, 2^31)");
  if (pdds_status e = check_csr(c, G, b)) return e;
  const int64_t kmax = c->k_max > 0 ? c->k_max : default_kmax(c, dt);
  c->st = pdds_stats_t{};
  c->timing_pending = false;
  int launches = 0;
  CK(c, cudaMemcpyAsync(G->row_ptr, c->d_row_ptr, (c->geo.n + 1) * 4, cudaMemcpyDeviceToDevice, s));
  CK(c, cudaMemcpyAsync(G->col, c->d_col, c->geo.nnz * 4, cudaMemcpyDeviceToDevice, s));
  CK(c, cudaMemsetAsync(G->val, 0, c->geo.nnz * 8, s));
  CK(c, cudaMemsetAsync(b, 0, c->geo.n * 8, s));
  CK(c, cudaMemsetAsync(c->d_scratch, 0, sizeof(pdds::Scratch), s));
  ProbDesc D = make_prob(c, (int)c->tag);
  D.Gval = G->val;
  D.b = b;
  D.n_per_knot = N;
  D.n_paths = Nu;
  if (N) {
    CK(c, pdds::launch_unit_prefix(N, c->geo.n, c->unit_paths, c->d_unit_prefix,
                                   c->d_path_prefix, &c->d_scratch->error, s));
    ++launches;
    D.knot_unit_prefix = c->d_unit_prefix;
    D.path_prefix = c->d_path_prefix;
  } else {
    D.units_per_knot = ceil_div(Nu, c->unit_paths);
  }
  CK(c, pdds::launch_prob_prefix_single(D, c->d_prob_prefix, s));
  ++launches;
  const bool gm = (scheme < 0 ? c->scheme : scheme) == PDDS_SCHEME_GM;
  const bool ext = gm || c->d_hknot != nullptr || c->interp == PDDS_INTERP_RBF;
  if (pdds_status e = run_paths(c, D, nullptr, 1, dt, seed, kmax,
                                reinterpret_cast<pdds::PathRecordDev*>(rec), s, stage_bytes(c),
                                c->geo.max_slots, c->tile_w, c->tile_h, c->coef_id, ext, gm,
                                reinterpret_cast<pdds::PathRecordDev*>(rec_gm)))
    return e;
  ++launches;
  CK(c, pdds::launch_finalize(G->row_ptr, G->col, G->val, b, N, Nu, c->geo.n, s));
  ++launches;
  c->st.kernel_launches = launches;
  c->timing_pending = c->timing;
  return PDDS_OK;
}

}  // namespace

namespace pdds {
void set_global_error(const std::string& msg) { g_last_error = msg; }
}  // namespace pdds

// ================================================================ C ABI
extern "C" {

pdds_status pdds_geometry_host(const pdds_grid* grid, int64_t* n, int64_t* nnz, double* xy,
                               int32_t* row_ptr, int32_t* col) {
  if (!grid) return fail(nullptr, PDDS_EINVAL, "geometry: grid is NULL");
  Geometry G;
  std::string err;
  if (!build_geometry(*grid, G, false, err)) return fail(nullptr, PDDS_EINVAL, err);
  if (n) *n = G.n;
  if (nnz) *nnz = G.nnz;
  if (xy)
    for (int64_t k = 0; k < G.n; ++k) {
      xy[2 * k] = grid->x0 + G.ki[k] * G.dx;
      xy[2 * k + 1] = grid->y0 + G.kj[k] * G.dy;
    }
  if (row_ptr) std::copy(G.row_ptr.begin(), G.row_ptr.end(), row_ptr);
  if (col) std::copy(G.col.begin(), G.col.end(), col);
  return PDDS_OK;
}

pdds_status pdds_create(const pdds_grid* grid, const pdds_coeffs* cf, pdds_ctx** out) {
  if (!grid || !cf || !out) return fail(nullptr, PDDS_EINVAL, "create: NULL argument");
  *out = nullptr;
  if (cf->kind != PDDS_COEF_BUILTIN || cf->builtin_id < 0 || cf->builtin_id > PDDS_COEF_POISSON_E1)
    return fail(nullptr, PDDS_EINVAL, "create: unknown coefficient set");
  auto* c = new (std::nothrow) pdds_ctx;
  if (!c) return fail(nullptr, PDDS_ENOMEM, "create: out of host memory");
  c->grid = *grid;
  c->coef_id = cf->builtin_id;
  std::memcpy(c->params, cf->params, sizeof(c->params));
  std::string err;
  if (!build_geometry(*grid, c->geo, true, err)) {
    free_ctx(c);
    return fail(nullptr, PDDS_EINVAL, err);
  }
  // c <= 0 (the setting of Eq. 6): the weight Y = exp(int c dt) stays <= 1,
  // which the exact 2^-30 fixed-point slot sums of the path kernel rely on
  if (c->coef_id == PDDS_COEF_CONSTANT && !(cf->params[3] <= 0)) {
    free_ctx(c);
    return fail(nullptr, PDDS_EINVAL, "create: CONSTANT needs params[3] (c) <= 0");
  }
  if (c->coef_id == PDDS_COEF_CONSTANT && !(std::fabs(cf->params[0]) > 0)) {
    free_ctx(c);
    return fail(nullptr, PDDS_EINVAL, "create: CONSTANT needs params[0] (sigma) != 0");
  }
  auto bail = [&](cudaError_t e, const char* what) {
    g_last_error = std::string("create: ") + what + ": " + cudaGetErrorString(e);
    free_ctx(c);
    return PDDS_ECUDA;
  };
  cudaError_t e;
  if ((e = cudaGetDevice(&c->device)) != cudaSuccess) return bail(e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device)) !=
      cudaSuccess)
    return bail(e, "multiprocessor count");
  const Geometry& G = c->geo;
  std::vector<float> sig_host, c_host;
  if (c->coef_id == PDDS_COEF_TABLE) {
    if (!cf->sigma_tab || !cf->c_tab || cf->tab_nx < 2 || cf->tab_ny < 2) {
      free_ctx(c);
      return fail(nullptr, PDDS_EINVAL, "create: TABLE needs sigma_tab, c_tab and tab_nx,ny >= 2");
    }
    c->tab_nx = cf->tab_nx;
    c->tab_ny = cf->tab_ny;
    const size_t cnt = (size_t)cf->tab_nx * cf->tab_ny;
    sig_host.resize(cnt);
    c_host.resize(cnt);
    if ((e = cudaMemcpy(sig_host.data(), cf->sigma_tab, cnt * 4, cudaMemcpyDefault)) != cudaSuccess)
      return bail(e, "sigma table copy");
    if ((e = cudaMemcpy(c_host.data(), cf->c_tab, cnt * 4, cudaMemcpyDefault)) != cudaSuccess)
      return bail(e, "c table copy");
    for (size_t i = 0; i < cnt; ++i) {
      // c <= 0 keeps Y <= 1 (exact fixed-point slot sums); s finite and nonzero
      if (!(c_host[i] <= 0.0f) || !std::isfinite(c_host[i]) || !std::isfinite(sig_host[i]) ||
          sig_host[i] == 0.0f) {
        free_ctx(c);
        return fail(nullptr, PDDS_EINVAL,
                    "create: TABLE needs every c_tab value finite and <= 0 and every sigma_tab "
                    "value finite and nonzero");
      }
    }
    // Tile covering every patch: nodes [i0, i0 + w) x [j0, j0 + h) with i0 a
    // multiple of 4 (16-byte TMA inner coordinate).
    const double tdx = (grid->x1 - grid->x0) / (cf->tab_nx - 1);
    const double tdy = (grid->y1 - grid->y0) / (cf->tab_ny - 1);
    int need_w = 0, need_h = 0;
    for (int64_t k = 0; k < G.n; ++k) {
      KnotDesc& d = c->geo.kd[k];
      const int pil = d.line[2], pih = d.line[0], pjl = d.line[3], pjh = d.line[1];
      const double fxl = pil * G.dx / tdx, fxh = pih * G.dx / tdx;
      const double fyl = pjl * G.dy / tdy, fyh = pjh * G.dy / tdy;
      const int i0 = ((int)std::floor(fxl + 1e-9) / 4) * 4;
      const int j0 = (int)std::floor(fyl + 1e-9);
      const int ihi = std::min((int)std::floor(fxh + 1e-9), cf->tab_nx - 2) + 1;
      const int jhi = std::min((int)std::floor(fyh + 1e-9), cf->tab_ny - 2) + 1;
      need_w = std::max(need_w, ihi - i0 + 1);
      need_h = std::max(need_h, jhi - j0 + 1);
      d.tile_i0 = i0;
      d.tile_j0 = j0;
      d.tab_fx = (float)(G.ki[k] * G.dx / tdx - i0);
      d.tab_fy = (float)(G.kj[k] * G.dy / tdy - j0);
    }
    c->tile_w = (int)round_up((size_t)need_w, 4);
    c->tile_h = need_h;
    // the TMA box holds 2 tile_w interleaved floats per row (<= 256)
    if (c->tile_w > 128 || c->tile_h > 256 || 2 * c->tile_w * c->tile_h * 4 > 96 * 1024) {
      free_ctx(c);
      return fail(nullptr, PDDS_EINVAL,
                  "create: coefficient tile per patch exceeds 128x256 nodes / 96 KB");
    }
    auto enc = get_encode_fn();
    if (!enc) {
      free_ctx(c);
      return fail(nullptr, PDDS_ECUDA, "create: cuTensorMapEncodeTiled unavailable");
    }
    // one table of interleaved (s, c) pairs per node, rows padded to 16 bytes
    const size_t pitch = round_up((size_t)2 * cf->tab_nx, 4);
    std::vector<float> padded(pitch * cf->tab_ny, 0.0f);
    for (int j = 0; j < cf->tab_ny; ++j)
      for (int i = 0; i < cf->tab_nx; ++i) {
        padded[j * pitch + 2 * i] = sig_host[(size_t)j * cf->tab_nx + i];
        padded[j * pitch + 2 * i + 1] = c_host[(size_t)j * cf->tab_nx + i];
      }
    if ((e = dalloc(&c->d_tab, padded.size())) != cudaSuccess) return bail(e, "table alloc");
    if ((e = cudaMemcpy(c->d_tab, padded.data(), padded.size() * 4, cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return bail(e, "table upload");
    CUtensorMap maps[1];
    {
      const cuuint64_t dims[2] = {(cuuint64_t)(2 * cf->tab_nx), (cuuint64_t)cf->tab_ny};
      const cuuint64_t strides[1] = {(cuuint64_t)(pitch * 4)};
      const cuuint32_t box[2] = {(cuuint32_t)(2 * c->tile_w), (cuuint32_t)c->tile_h};
      const cuuint32_t es[2] = {1, 1};
      CUresult r = enc(&maps[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->d_tab, dims, strides, box,
                       es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) {
        free_ctx(c);
        return fail(nullptr, PDDS_ECUDA, "create: cuTensorMapEncodeTiled failed");
      }
    }
    if ((e = cudaMalloc(reinterpret_cast<void**>(&c->d_tmap), sizeof(maps))) != cudaSuccess)
      return bail(e, "tensor map alloc");
    if ((e = cudaMemcpy(c->d_tmap, maps, sizeof(maps), cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(e, "tensor map upload");
  }
  sigma_bounds(*cf, sig_host, c->s_min, c->s_max);
  const int64_t n = G.n;
  if ((e = dalloc(&c->d_knots, n)) != cudaSuccess) return bail(e, "knot table alloc");
  if ((e = dalloc(&c->d_slot2csr, G.slot2csr.size())) != cudaSuccess) return bail(e, "slot alloc");
  if ((e = dalloc(&c->d_row_ptr, n + 1)) != cudaSuccess) return bail(e, "row_ptr alloc");
  if ((e = dalloc(&c->d_col, G.nnz)) != cudaSuccess) return bail(e, "col alloc");
  if ((e = dalloc(&c->d_scratch, 1)) != cudaSuccess) return bail(e, "scratch alloc");
  if ((e = dalloc(&c->d_unit_prefix, n + 1)) != cudaSuccess) return bail(e, "prefix alloc");
  if ((e = dalloc(&c->d_path_prefix, n + 1)) != cudaSuccess) return bail(e, "prefix alloc");
  if ((e = dalloc(&c->d_prob_prefix, 2)) != cudaSuccess) return bail(e, "prefix alloc");
  if ((e = cudaMemcpy(c->d_knots, G.kd.data(), n * sizeof(KnotDesc), cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return bail(e, "knot upload");
  if ((e = cudaMemcpy(c->d_slot2csr, G.slot2csr.data(), G.slot2csr.size() * 4,
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(e, "slot upload");
  if ((e = cudaMemcpy(c->d_row_ptr, G.row_ptr.data(), (n + 1) * 4, cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return bail(e, "row_ptr upload");
  if ((e = cudaMemcpy(c->d_col, G.col.data(), G.nnz * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(e, "col upload");
  if ((e = cudaEventCreate(&c->ev0)) != cudaSuccess) return bail(e, "event");
  if ((e = cudaEventCreate(&c->ev1)) != cudaSuccess) return bail(e, "event");
  // Distinct interface-stencil lengths per orientation (0: lines along x, the
  // N/S sides; 1: along y, the E/W sides), kept for the RBF tables.
  for (const KnotDesc& d : G.kd)
    for (int o = 0; o < 4; ++o) {
      if ((d.dirbits >> o) & 1) continue;
      const int L = d.b[o] - d.a[o] + 1;
      std::vector<int>& v = c->stencil_len[(o == 0 || o == 2) ? 1 : 0];
      if (std::find(v.begin(), v.end(), L) == v.end()) v.push_back(L);
    }
  // Knot data on the host is only needed for coordinates from here on.
  c->geo.kd.clear();
  c->geo.kd.shrink_to_fit();
  c->geo.slot2csr.clear();
  c->geo.slot2csr.shrink_to_fit();
  *out = c;
  return PDDS_OK;
}

void pdds_destroy(pdds_ctx* c) {
  if (c) cudaDeviceSynchronize();
  free_ctx(c);
}

pdds_status pdds_num_knots(const pdds_ctx* c, int64_t* n, int64_t* nnz) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "num_knots: NULL context");
  if (n) *n = c->geo.n;
  if (nnz) *nnz = c->geo.nnz;
  return PDDS_OK;
}

pdds_status pdds_knot_coords(const pdds_ctx* c, double* xy) {
  if (!c || !xy) return fail(nullptr, PDDS_EINVAL, "knot_coords: NULL argument");
  for (int64_t k = 0; k < c->geo.n; ++k) {
    xy[2 * k] = c->grid.x0 + c->geo.ki[k] * c->geo.dx;
    xy[2 * k + 1] = c->grid.y0 + c->geo.kj[k] * c->geo.dy;
  }
  return PDDS_OK;
}

pdds_status pdds_set_step_cap(pdds_ctx* c, int64_t k_max) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "set_step_cap: NULL context");
  if (k_max < 0 || k_max >= ((int64_t)1 << 31))
    return fail(c, PDDS_EINVAL, "set_step_cap: need 0 <= k_max < 2^31");
  c->k_max = k_max;
  return PDDS_OK;
}

pdds_status pdds_set_launch(pdds_ctx* c, int32_t block, int32_t per_sm, int32_t unit_paths,
                            int32_t exit_batch) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "set_launch: NULL context");
  if (block && (block < 64 || block > 1024 || block % 32))
    return fail(c, PDDS_EINVAL, "set_launch: block must be a multiple of 32 in [64, 1024]");
  if (per_sm < 0 || per_sm > 32) return fail(c, PDDS_EINVAL, "set_launch: ctas_per_sm in [0, 32]");
  if (unit_paths && (unit_paths < 32 || unit_paths > (1 << 24)))
    return fail(c, PDDS_EINVAL, "set_launch: unit_paths in [32, 2^24]");
  if (exit_batch && (exit_batch < 1 || exit_batch > 32))
    return fail(c, PDDS_EINVAL, "set_launch: exit_batch in [1, 32]");
  if (block) c->block = block;
  c->ctas_per_sm = per_sm;
  if (unit_paths) c->unit_paths = unit_paths;
  if (exit_batch) c->exit_batch = exit_batch;
  return PDDS_OK;
}

pdds_status pdds_get_launch(const pdds_ctx* c, int32_t* block, int32_t* per_sm,
                            int32_t* unit_paths, int32_t* exit_batch) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "get_launch: NULL context");
  if (block) *block = c->block;
  if (per_sm) *per_sm = c->ctas_per_sm;
  if (unit_paths) *unit_paths = (int32_t)c->unit_paths;
  if (exit_batch) *exit_batch = c->exit_batch;
  return PDDS_OK;
}

pdds_status pdds_boundary_samples(const pdds_ctx* c, int32_t n_per_side, float* xy, float* g,
                                  void* stream) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "boundary_samples: NULL context");
  if (n_per_side < 1 || n_per_side > (1 << 26) || !xy || !g)
    return fail(const_cast<pdds_ctx*>(c), PDDS_EINVAL,
                "boundary_samples: need 1 <= n_per_side <= 2^26 and device xy, g");
  (void)cudaGetLastError();
  const double dom[4] = {c->grid.x0, c->grid.x1, c->grid.y0, c->grid.y1};
  CK(const_cast<pdds_ctx*>(c), pdds::launch_boundary_samples(c->coef_id, dom, c->params, n_per_side,
                                                               xy, g, (cudaStream_t)stream));
  return PDDS_OK;
}

pdds_status pdds_set_philox_tag(pdds_ctx* c, uint32_t tag) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "set_philox_tag: NULL context");
  c->tag = tag;
  return PDDS_OK;
}

pdds_status pdds_set_network_engine(pdds_ctx* c, int32_t engine) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "set_network_engine: NULL context");
  if (engine != PDDS_NET_MMA_SYNC && engine != PDDS_NET_TCGEN05)
    return fail(c, PDDS_EINVAL, "set_network_engine: unknown engine");
  c->net_engine = engine;
  return PDDS_OK;
}

pdds_status pdds_set_wait_limit(pdds_ctx* c, double seconds) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "set_wait_limit: NULL context");
  if (!(seconds >= 0) || seconds > 1e6) return fail(c, PDDS_EINVAL, "set_wait_limit: need 0 <= s <= 1e6");
  c->wait_s = seconds;
  return PDDS_OK;
}

pdds_status pdds_autotune(pdds_ctx* c, int64_t n_paths, double dt, uint64_t seed,
                          void* stream) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "autotune: NULL context");
  if (n_paths < 1 || !(dt > 0)) return fail(c, PDDS_EINVAL, "autotune: need n_paths >= 1, dt > 0");
  // Cache key: device, coefficient set, control variate, grid shape, budget.
  struct Key {
    int dev, coef, cv, xk, Hx, Hy, m, ext;
    int64_t N;
    bool operator<(const Key& o) const {
      return std::tie(dev, coef, cv, xk, Hx, Hy, m, ext, N) <
             std::tie(o.dev, o.coef, o.cv, o.xk, o.Hx, o.Hy, o.m, o.ext, o.N);
    }
  };
  struct Shape { int block, unit, batch; };
  static std::mutex mu;
  static std::map<Key, Shape> cache;
  // xk: the extended-exit kernel (GM scheme or per-knot steps) is a different kernel
  const int xk = (c->scheme == PDDS_SCHEME_GM ? 1 : 0) + (c->d_hknot ? 2 : 0);
  // the in-path network on tcgen05 is its own kernel too
  const bool net_tc = c->cv_mode == 1 && c->net_engine == PDDS_NET_TCGEN05;
  const Key key{c->device, c->coef_id, net_tc ? 3 : c->cv_mode, xk, c->grid.Hx, c->grid.Hy,
                c->grid.m, c->grid.ext, n_paths};
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      c->block = it->second.block;
      c->unit_paths = it->second.unit;
      c->exit_batch = it->second.batch;
      c->ctas_per_sm = 0;
      return PDDS_OK;
    }
  }
  (void)cudaGetLastError();
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = c->geo.n, nnz = c->geo.nnz;
  // Stage 1 sample: every k-th knot at the full budget (others get none), k >= 8
  // and large enough that the sample has at most 2e8 paths; the finalists run on
  // the whole problem, or on every k2-th knot when it has more than 1e9 paths.
  const int64_t total = n * n_paths;
  const int64_t k1 = std::max<int64_t>(8, (total + 199999999) / 200000000);
  const int64_t k2 = std::max<int64_t>(1, (total + 999999999) / 1000000000);
  std::vector<int64_t> Nh(n, 0), Nf(n, 0);
  for (int64_t k = 0; k < n; k += k1) Nh[k] = n_paths;
  for (int64_t k = 0; k < n; k += k2) Nf[k] = n_paths;
  int64_t *dN = nullptr, *dF = nullptr;
  int32_t *rp = nullptr, *col = nullptr;
  double *val = nullptr, *b = nullptr;
  auto cleanup = [&] {
    cudaFree(dN); cudaFree(dF); cudaFree(rp); cudaFree(col); cudaFree(val); cudaFree(b);
  };
  if (dalloc(&dN, n) || dalloc(&dF, n) || dalloc(&rp, n + 1) || dalloc(&col, nnz) ||
      dalloc(&val, nnz) || dalloc(&b, n)) {
    cleanup();
    return fail(c, PDDS_ENOMEM, "autotune: scratch allocation failed");
  }
  pdds_csr G{n, nnz, rp, col, val};
  pdds_status st = PDDS_OK;
  if (cudaMemcpy(dN, Nh.data(), n * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dF, Nf.data(), n * 8, cudaMemcpyHostToDevice) != cudaSuccess)
    st = fail(c, PDDS_ECUDA, "autotune: upload failed");
  const bool timing = c->timing;
  // Short paths (few steps per exit) favour small CTAs and units: all warps of a
  // CTA refill from its two staged units, so large CTAs contend on them.
  const int blocks[] = {64, 128, 256, 512};
  const int units[] = {256, 1024, 4096, 16384};
  const int batches[] = {2, 4, 8, 16};
  Shape best{c->block, (int)c->unit_paths, c->exit_batch};
  c->timing = true;
  c->ctas_per_sm = 0;
  std::vector<Shape> shapes;
  for (int bl : blocks)
    for (int un : units)
      for (int ba : batches)
        if (!(c->cv_mode == 1 && bl > 256) && !(net_tc && bl != 128))
          shapes.push_back(Shape{bl, un, ba});
  auto time_shape = [&](const Shape& sh, const int64_t* N, int64_t Nu, float& ms) {
    c->block = sh.block;
    c->unit_paths = sh.unit;
    c->exit_batch = sh.batch;
    st = assemble_impl(c, N, Nu, dt, seed, &G, b, nullptr, s);
    if (st == PDDS_OK) st = read_timing(c);
    if (st == PDDS_OK) ms = std::min(ms, c->st.path_kernel_ms);
  };
  // first pass: every shape once on the sample; second pass: the best twelve again
  // (a few-millisecond timing is noisy at the 2-3 % that separates the best)
  std::vector<float> ms(shapes.size(), 1e30f);
  for (size_t i = 0; i < shapes.size() && st == PDDS_OK; ++i) time_shape(shapes[i], dN, 0, ms[i]);
  std::vector<size_t> order(shapes.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  auto by_ms = [&](size_t a, size_t b2) { return ms[a] < ms[b2]; };
  std::stable_sort(order.begin(), order.end(), by_ms);
  for (size_t f = 0; f < std::min<size_t>(12, order.size()) && st == PDDS_OK; ++f)
    time_shape(shapes[order[f]], dN, 0, ms[order[f]]);
  std::stable_sort(order.begin(), order.end(), by_ms);
  // The sample's tail (few units left, lanes idle) weighs more than in the
  // full problem, so the three best are timed twice more on the large sample.
  const size_t finalists = std::min<size_t>(3, order.size());
  std::vector<float> full(finalists, 1e30f);
  for (int round = 0; round < 2 && st == PDDS_OK; ++round)
    for (size_t f = 0; f < finalists && st == PDDS_OK; ++f) {
      if (k2 == 1) time_shape(shapes[order[f]], nullptr, n_paths, full[f]);
      else time_shape(shapes[order[f]], dF, 0, full[f]);
    }
  float best_ms = 1e30f;
  for (size_t f = 0; f < finalists; ++f)
    if (full[f] < best_ms) {
      best_ms = full[f];
      best = shapes[order[f]];
    }
  c->timing = timing;
  c->block = best.block;
  c->unit_paths = best.unit;
  c->exit_batch = best.batch;
  cleanup();
  if (st != PDDS_OK) return st;
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = best;
  return PDDS_OK;
}

pdds_status pdds_set_control_variate(pdds_ctx* c, const float* theta) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "set_control_variate: NULL context");
  if (!theta) {
    c->cv_mode = 0;
    return PDDS_OK;
  }
  if (!pdds::path_kernel_has_cv(c->coef_id))
    return fail(c, PDDS_EINVAL, "set_control_variate: not available for this coefficient set");
  (void)cudaGetLastError();
  c->cv_mode = 0;  // detached until the new network is staged (a failure leaves none)
  if (!c->d_mlp) CK(c, cudaMalloc(&c->d_mlp, pdds::mlp_image_bytes()));
  CK(c, pdds::mlp_stage(theta, c->d_mlp, nullptr));
  CK(c, cudaDeviceSynchronize());
  {
    // host copy of the FP32 vectors (kernel parameter of the tcgen05 engine)
    std::vector<float> th(PDDS_MLP_NPARAM);
    CK(c, cudaMemcpy(th.data(), theta, sizeof(float) * PDDS_MLP_NPARAM, cudaMemcpyDefault));
    for (int u = 0; u < 64; ++u) {
      c->net_w[u] = th[2 * u];
      c->net_w[64 + u] = th[2 * u + 1];
      c->net_w[128 + u] = th[128 + u];   // b1
      c->net_w[192 + u] = th[4288 + u];  // b2
      c->net_w[256 + u] = th[4352 + u];  // w3
    }
  }
  c->cv_mode = 1;
  return PDDS_OK;
}

pdds_status pdds_set_control_variate_grid(pdds_ctx* c, const float* grad_xy, int32_t nx,
                                          int32_t ny) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "set_control_variate_grid: NULL context");
  if (!grad_xy) {
    c->cv_mode = 0;
    return PDDS_OK;
  }
  if (nx < 2 || ny < 2 || (int64_t)nx * ny > ((int64_t)1 << 28))
    return fail(c, PDDS_EINVAL, "set_control_variate_grid: need 2 <= nx, ny and nx*ny <= 2^28");
  (void)cudaGetLastError();
  c->cv_mode = 0;  // detached until the new table is built (a failure leaves none)
  const size_t count = (size_t)nx * ny * 2;
  const size_t cells = (size_t)(nx - 1) * (ny - 1) * 8;
  if (c->cv_nx != nx || c->cv_ny != ny) {
    CK(c, cudaFree(c->d_cvtab));
    c->d_cvtab = nullptr;
    c->cv_nx = c->cv_ny = 0;
    if (dalloc(&c->d_cvtab, cells) != cudaSuccess)
      return fail(c, PDDS_ENOMEM, "set_control_variate_grid: table allocation failed");
  }
  float* nodes = nullptr;
  if (dalloc(&nodes, count) != cudaSuccess)
    return fail(c, PDDS_ENOMEM, "set_control_variate_grid: node staging allocation failed");
  cudaError_t e = cudaMemcpy(nodes, grad_xy, count * 4, cudaMemcpyDefault);
  if (e == cudaSuccess) e = pdds::launch_cv_cells(nodes, nx, ny, c->d_cvtab, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(nodes);
  CK(c, e);
  c->cv_nx = nx;
  c->cv_ny = ny;
  c->cv_mode = 2;
  return PDDS_OK;
}

pdds_status pdds_set_timing(pdds_ctx* c, int32_t on) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "set_timing: NULL context");
  c->timing = on != 0;
  return PDDS_OK;
}

pdds_status pdds_set_scheme(pdds_ctx* c, int32_t scheme) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "set_scheme: NULL context");
  if (scheme != PDDS_SCHEME_EM && scheme != PDDS_SCHEME_GM)
    return fail(c, PDDS_EINVAL, "set_scheme: scheme must be PDDS_SCHEME_EM or PDDS_SCHEME_GM");
  c->scheme = scheme;
  return PDDS_OK;
}

pdds_status pdds_set_knot_steps(pdds_ctx* c, const double* h) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "set_knot_steps: NULL context");
  (void)cudaGetLastError();
  if (!h) {
    CK(c, cudaFree(c->d_hknot));
    c->d_hknot = nullptr;
    c->h_min = 0;
    return PDDS_OK;
  }
  const int64_t n = c->geo.n;
  std::vector<double> hh(n);
  CK(c, cudaMemcpy(hh.data(), h, n * 8, cudaMemcpyDefault));
  double lo = 1e300;
  for (double v : hh) {
    if (!(v > 0) || !std::isfinite(v))
      return fail(c, PDDS_EINVAL, "set_knot_steps: every h_k must be finite and > 0");
    lo = std::min(lo, v);
  }
  if (!c->d_hknot) CK(c, dalloc(&c->d_hknot, n));
  CK(c, cudaMemcpy(c->d_hknot, hh.data(), n * 8, cudaMemcpyHostToDevice));
  c->h_min = lo;
  return PDDS_OK;
}

pdds_status pdds_set_interpolation(pdds_ctx* c, int32_t kind, double shape, double* shape_used,
                                   double* table_err) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "set_interpolation: NULL context");
  (void)cudaGetLastError();
  if (kind == PDDS_INTERP_LINEAR) {
    c->interp = kind;
    if (shape_used) *shape_used = 0;
    if (table_err) *table_err = 0;
    return PDDS_OK;
  }
  if (kind != PDDS_INTERP_RBF)
    return fail(c, PDDS_EINVAL, "set_interpolation: kind must be PDDS_INTERP_LINEAR or _RBF");
  if (!std::isfinite(shape)) return fail(c, PDDS_EINVAL, "set_interpolation: shape not finite");
  // stencil lengths per orientation (0: lines along x, sides N/S; 1: along y, E/W)
  const std::vector<int>* len = c->stencil_len;
  int lmax_any = 0;
  for (int o = 0; o < 2; ++o)
    for (int L : len[o]) lmax_any = std::max(lmax_any, L);
  if (lmax_any < 2) return fail(c, PDDS_EINVAL, "set_interpolation: no interface stencils");
  const double sp[2] = {c->geo.dx, c->geo.dy};
  double cabs = shape;
  if (!(cabs > 0)) {
    // Sec. 5.1: c such that cond(Phi) of the longest stencil is 1e10
    cabs = pdds::rbf_shape_for_cond(lmax_any, 1e10) * std::min(sp[0], sp[1]);
  }
  const double c_lat[2] = {cabs / sp[0], cabs / sp[1]};
  pdds::RbfTables T;
  std::string err;
  if (!pdds::rbf_build_tables(len, c_lat, T, err)) return fail(c, PDDS_EINVAL, "set_interpolation: " + err);
  float* coef = nullptr;
  int64_t* off = nullptr;
  if (dalloc(&coef, T.coef.size()) != cudaSuccess || dalloc(&off, T.offset.size()) != cudaSuccess) {
    cudaFree(coef);
    cudaFree(off);
    return fail(c, PDDS_ENOMEM, "set_interpolation: table allocation failed");
  }
  CK(c, cudaMemcpy(coef, T.coef.data(), T.coef.size() * 4, cudaMemcpyHostToDevice));
  CK(c, cudaMemcpy(off, T.offset.data(), T.offset.size() * 8, cudaMemcpyHostToDevice));
  cudaFree(c->d_rbf_coef);
  cudaFree(c->d_rbf_off);
  c->d_rbf_coef = coef;
  c->d_rbf_off = off;
  c->rbf_deg = T.degree;
  c->rbf_lmax = T.lmax;
  c->rbf_shape = cabs;
  c->interp = PDDS_INTERP_RBF;
  if (shape_used) *shape_used = cabs;
  if (table_err) *table_err = T.max_err;
  return PDDS_OK;
}

pdds_status pdds_calibrate(pdds_ctx* c, const double* u0, const int64_t* N, int64_t Nu, double dt,
                           uint64_t seed, double* moments, void* stream) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "calibrate: NULL context");
  if (!u0 || !moments) return fail(c, PDDS_EINVAL, "calibrate: u0 and moments are required");
  (void)cudaGetLastError();
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = c->geo.n, nnz = c->geo.nnz;
  // records per pass: sum of N_k
  int64_t total = 0;
  if (N) {
    std::vector<int64_t> Nh(n);
    CK(c, cudaMemcpyAsync(Nh.data(), N, n * 8, cudaMemcpyDefault, s));
    CK(c, cudaStreamSynchronize(s));
    for (int64_t v : Nh) {
      if (v < 0 || v >= ((int64_t)1 << 31))
        return fail(c, PDDS_EINVAL, "calibrate: every N_k must be in [0, 2^31)");
      total += v;
    }
  } else {
    if (Nu < 1 || Nu >= ((int64_t)1 << 31))
      return fail(c, PDDS_EINVAL, "calibrate: n_paths must be in [1, 2^31)");
    total = Nu * n;
  }
  if (total > c->cal_rec_cap) {
    CK(c, cudaFree(c->cal_rec));
    c->cal_rec = nullptr;
    c->cal_rec_cap = 0;
    if (dalloc(&c->cal_rec, 2 * (size_t)std::max<int64_t>(total, 1)) != cudaSuccess)
      return fail(c, PDDS_ENOMEM, "calibrate: record scratch allocation failed");
    c->cal_rec_cap = total;
  }
  if (!c->cal_val) {
    if (dalloc(&c->cal_val, nnz) || dalloc(&c->cal_b, n) || dalloc(&c->cal_rp, n + 1) ||
        dalloc(&c->cal_col, nnz))
      return fail(c, PDDS_ENOMEM, "calibrate: CSR scratch allocation failed");
  }
  pdds_csr G{n, nnz, c->cal_rp, c->cal_col, c->cal_val};
  pdds_path_record* rec_em = c->cal_rec;
  pdds_path_record* rec_gm = c->cal_rec + c->cal_rec_cap;
  // One pass of the mixed trajectory of Sec. 4.1: each path records its first
  // step beyond a moved side (GM), then steps on to its first step outside
  // the patch (naive), which is recorded and accumulated -- the naive run's
  // paths, the GM exits on the way.
  if (pdds_status e = assemble_impl(c, N, Nu, dt, seed, &G, c->cal_b, rec_em, s,
                                    PDDS_SCHEME_GM, rec_gm))
    return e;
  CK(c, pdds::launch_calib_moments(reinterpret_cast<const pdds::PathRecordDev*>(rec_em),
                                   reinterpret_cast<const pdds::PathRecordDev*>(rec_gm),
                                   N ? c->d_path_prefix : nullptr, Nu, u0, n, moments,
                                   make_prob(c, 0), s));
  CK(c, cudaStreamSynchronize(s));
  c->st.kernel_launches += 1;
  return PDDS_OK;
}

pdds_status pdds_plan(const double* moments, int64_t n, double eps, double h0, double h0p,
                      int64_t n_job, double* h_out, int64_t* n_out, double* diag, void* stream) {
  (void)cudaGetLastError();
  if (!moments || !h_out || !n_out)
    return fail(nullptr, PDDS_EINVAL, "plan: moments, h_out and n_out are required");
  if (n < 1 || !(eps > 0) || !(h0 > 0) || !(h0p > 0) || n_job < 1 || n_job > 0x7fffffffll ||
      !std::isfinite(eps) || !std::isfinite(h0) || !std::isfinite(h0p))
    return fail(nullptr, PDDS_EINVAL, "plan: need n >= 1, eps, h0, h0' > 0 and 1 <= N_job < 2^31");
  cudaError_t e = pdds::launch_plan(moments, n, eps, h0, h0p, n_job, h_out, n_out, diag,
                                    (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(nullptr, PDDS_ECUDA, std::string("plan: ") + cudaGetErrorString(e));
  return PDDS_OK;
}

pdds_status pdds_assemble(pdds_ctx* c, const int64_t* N, int64_t Nu, double dt, uint64_t seed,
                          pdds_csr* G, double* b, void* stream) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "assemble: NULL context");
  return assemble_impl(c, N, Nu, dt, seed, G, b, nullptr, (cudaStream_t)stream);
}

pdds_status pdds_assemble_records(pdds_ctx* c, const int64_t* N, int64_t Nu, double dt,
                                  uint64_t seed, pdds_csr* G, double* b, pdds_path_record* rec,
                                  void* stream) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "assemble_records: NULL context");
  if (!rec) return fail(c, PDDS_EINVAL, "assemble_records: records is NULL");
  return assemble_impl(c, N, Nu, dt, seed, G, b, rec, (cudaStream_t)stream);
}

pdds_status pdds_stats(pdds_ctx* c, pdds_stats_t* out) {
  if (!c || !out) return fail(nullptr, PDDS_EINVAL, "stats: NULL argument");
  pdds::Scratch s{};
  CK(c, cudaDeviceSynchronize());
  CK(c, cudaMemcpy(&s, c->d_scratch, sizeof(s), cudaMemcpyDeviceToHost));
  if (pdds_status e = read_timing(c)) return e;
  c->st.path_steps = (int64_t)s.steps;
  c->st.paths = (int64_t)s.paths;
  c->st.truncated = (int64_t)s.truncated;
  c->st.clamped = (int64_t)s.clamped;
  c->st.units = (int64_t)s.units;
  c->st.device_error = s.error;
  *out = c->st;
  return s.error ? (pdds_status)s.error : PDDS_OK;
}

const char* pdds_last_error(const pdds_ctx* c) {
  return c ? c->err.c_str() : g_last_error.c_str();
}

pdds_status pdds_solve(pdds_ctx* c, const pdds_csr* G, const double* b, double* u,
                       double rtol, int32_t maxit, int32_t* iters, void* stream) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "solve: NULL context");
  if (!G || !b || !u || !G->row_ptr || !G->col || !G->val)
    return fail(c, PDDS_EINVAL, "solve: NULL matrix/vector");
  if (G->n != c->geo.n || G->nnz != c->geo.nnz)
    return fail(c, PDDS_EINVAL, "solve: G sized differently from pdds_num_knots");
  if (!(rtol > 0) || maxit < 1) return fail(c, PDDS_EINVAL, "solve: need rtol > 0, maxit >= 1");
  (void)cudaGetLastError();
  const int64_t n = c->geo.n;
  if (!c->d_work) {
    CK(c, dalloc(&c->d_work, pdds::bicgstab_work_doubles(n)));
    CK(c, cudaMalloc(reinterpret_cast<void**>(&c->d_scalars), pdds::bicgstab_scalars_bytes()));
  }
  int32_t it = 0;
  double rel = 0;
  int conv = 0, nl = 0;
  CK(c, pdds::bicgstab_device(G->row_ptr, G->col, G->val, b, u, n, c->d_work, c->d_scalars, rtol,
                              maxit, &it, &rel, &conv, &nl, (cudaStream_t)stream));
  c->st.solve_iters = it;
  c->st.solve_relres = rel;
  c->st.kernel_launches += nl;
  if (iters) *iters = it;
  if (conv != 1) {
    char buf[200];
    std::snprintf(buf, sizeof buf, "solve: no convergence after %d iterations (relres %.3e)%s",
                  it, rel, pdds::bicgstab_stop_reason(conv));
    return fail(c, PDDS_ENOCONV, buf);
  }
  return PDDS_OK;
}

pdds_status pdds_assemble_solve_host(pdds_ctx* c, const int64_t* N_host, int64_t Nu, double dt,
                                     uint64_t seed, double rtol, int32_t maxit, int32_t* rp_host,
                                     int32_t* col_host, double* val_host, double* b_host,
                                     double* u_host, void* stream) {
  if (!c) return fail(nullptr, PDDS_EINVAL, "assemble_solve_host: NULL context");
  if (!val_host || !b_host || !u_host)
    return fail(c, PDDS_EINVAL, "assemble_solve_host: val, b and u host buffers are required");
  const int64_t n = c->geo.n, nnz = c->geo.nnz;
  for (int64_t k = 0; N_host && k < n; ++k)
    if (N_host[k] < 0 || N_host[k] > 0x7fffffffll)
      return fail(c, PDDS_EINVAL, "assemble_solve_host: every N_k must be in [0, 2^31)");
  cudaStream_t s = (cudaStream_t)stream;
  if (!c->e_rp) {
    CK(c, dalloc(&c->e_N, n));
    CK(c, dalloc(&c->e_rp, n + 1));
    CK(c, dalloc(&c->e_col, nnz));
    CK(c, dalloc(&c->e_val, nnz));
    CK(c, dalloc(&c->e_b, n));
    CK(c, dalloc(&c->e_u, n));
  }
  if (N_host) CK(c, cudaMemcpyAsync(c->e_N, N_host, n * 8, cudaMemcpyHostToDevice, s));
  pdds_csr G{n, nnz, c->e_rp, c->e_col, c->e_val};
  if (pdds_status e = assemble_impl(c, N_host ? c->e_N : nullptr, Nu, dt, seed, &G, c->e_b,
                                    nullptr, s))
    return e;
  const int launches = c->st.kernel_launches;
  pdds_status se = pdds_solve(c, &G, c->e_b, c->e_u, rtol, maxit, nullptr, stream);
  if (se != PDDS_OK && se != PDDS_ENOCONV) return se;
  (void)launches;
  if (rp_host) CK(c, cudaMemcpyAsync(rp_host, c->e_rp, (n + 1) * 4, cudaMemcpyDeviceToHost, s));
  if (col_host) CK(c, cudaMemcpyAsync(col_host, c->e_col, nnz * 4, cudaMemcpyDeviceToHost, s));
  CK(c, cudaMemcpyAsync(val_host, c->e_val, nnz * 8, cudaMemcpyDeviceToHost, s));
  CK(c, cudaMemcpyAsync(b_host, c->e_b, n * 8, cudaMemcpyDeviceToHost, s));
  CK(c, cudaMemcpyAsync(u_host, c->e_u, n * 8, cudaMemcpyDeviceToHost, s));
  CK(c, cudaStreamSynchronize(s));
  return se;
}

pdds_status pdds_assemble_batch(pdds_ctx* const* ctxs, int32_t count,
                                const int64_t* const* N, int64_t Nu, double dt, uint64_t seed,
                                pdds_csr* const* G, double* const* b, void* stream) {
  if (!ctxs || count < 1 || !ctxs[0] || !G || !b)
    return fail(nullptr, PDDS_EINVAL, "assemble_batch: need count >= 1 contexts, G and b");
  pdds_ctx* c0 = ctxs[0];
  (void)cudaGetLastError();
  if (!(dt > 0)) return fail(c0, PDDS_EINVAL, "assemble_batch: dt must be > 0");
  int max_slots = 0, tw = 0, th = 0;
  int64_t kmax = 0;
  double dom_bound = 0.0;  // max |coordinate| over the batch's domains
  for (int i = 0; i < count; ++i) {
    pdds_ctx* c = ctxs[i];
    if (!c) return fail(c0, PDDS_EINVAL, "assemble_batch: NULL context in the list");
    dom_bound = std::max({dom_bound, std::fabs(c->grid.x0), std::fabs(c->grid.x1),
                          std::fabs(c->grid.y0), std::fabs(c->grid.y1)});
    if (c->coef_id != c0->coef_id)
      return fail(c0, PDDS_EINVAL, "assemble_batch: all problems need the same coefficient set");
    if (c->device != c0->device)
      return fail(c0, PDDS_EINVAL, "assemble_batch: all problems need the same device");
    if (c->cv_mode)
      return fail(c0, PDDS_EINVAL, "assemble_batch: control variates are not supported in batches");
    if (c->scheme != PDDS_SCHEME_EM || c->d_hknot || c->interp != PDDS_INTERP_LINEAR)
      return fail(c0, PDDS_EINVAL,
                  "assemble_batch: the Gobet-Menozzi scheme, per-knot steps and RBF stencils "
                  "are not supported in batches");
    if (pdds_status e = check_csr(c, G[i], b[i])) return fail(c0, e, c->err);
    if (!(N && N[i]) && (Nu < 1 || Nu >= ((int64_t)1 << 31)))
      return fail(c0, PDDS_EINVAL, "assemble_batch: n_paths must be in [1, 2^31)");
    max_slots = std::max(max_slots, c->geo.max_slots);
    tw = std::max(tw, c->tile_w);
    th = std::max(th, c->tile_h);
    kmax = std::max(kmax, c->k_max > 0 ? c->k_max : default_kmax(c, dt));
  }
  c0->dom_bound_all = dom_bound;
  cudaStream_t s = (cudaStream_t)stream;
  // Graph key: everything the captured sequence depends on.
  std::vector<uint64_t> key = {(uint64_t)count, (uint64_t)Nu, (uint64_t)seed, (uint64_t)kmax,
                               (uint64_t)c0->block, (uint64_t)c0->ctas_per_sm,
                               (uint64_t)c0->unit_paths, (uint64_t)c0->exit_batch};
  uint64_t dtb;
  std::memcpy(&dtb, &dt, 8);
  key.push_back(dtb);
  for (int i = 0; i < count; ++i) {
    key.push_back((uint64_t)(uintptr_t)ctxs[i]);
    key.push_back((uint64_t)(uintptr_t)(N ? N[i] : nullptr));
    key.push_back((uint64_t)(uintptr_t)G[i]->val);
    key.push_back((uint64_t)(uintptr_t)G[i]->row_ptr);
    key.push_back((uint64_t)(uintptr_t)G[i]->col);
    key.push_back((uint64_t)(uintptr_t)b[i]);
  }
  if (!(c0->graph && key == c0->graph_key)) {
    if (c0->graph) { cudaGraphExecDestroy(c0->graph); c0->graph = nullptr; }
    std::vector<ProbDesc> probs(count);
    for (int i = 0; i < count; ++i) {
      pdds_ctx* c = ctxs[i];
      ProbDesc D = make_prob(c, i);
      D.Gval = G[i]->val;
      D.b = b[i];
      D.n_per_knot = N ? N[i] : nullptr;
      D.n_paths = Nu;
      if (D.n_per_knot) {
        D.knot_unit_prefix = c->d_unit_prefix;
        D.path_prefix = c->d_path_prefix;
      } else {
        D.units_per_knot = ceil_div(Nu, c0->unit_paths);
      }
      probs[i] = D;
    }
    if (c0->batch_cap < count) {
      cudaFree(c0->d_batch);
      c0->d_batch = nullptr;
      CK(c0, dalloc(&c0->d_batch, count));
      cudaFree(c0->d_prob_prefix);
      c0->d_prob_prefix = nullptr;
      CK(c0, dalloc(&c0->d_prob_prefix, count + 1));
      c0->batch_cap = count;
    }
    CK(c0, cudaStreamSynchronize(s));  // a previous replay may still read the old table
    CK(c0, cudaMemcpy(c0->d_batch, probs.data(), count * sizeof(ProbDesc), cudaMemcpyHostToDevice));
    const size_t sb = [&] {
      size_t x = pdds::stage_header_bytes() + round_up((size_t)max_slots * 8, 128);
      if (c0->coef_id == PDDS_COEF_TABLE) x += round_up((size_t)2 * tw * th * 4, 128);
      return round_up(x, 128);
    }();
    CK(c0, pdds::set_path_kernel_smem(c0->coef_id, false, 0, false, 2 * sb));
    // Capture on a private non-blocking stream (the legacy default stream
    // cannot be captured); the instantiated graph is launched on the caller's.
    if (!c0->cap_stream) CK(c0, cudaStreamCreateWithFlags(&c0->cap_stream, cudaStreamNonBlocking));
    const cudaStream_t user_stream = s;
    (void)user_stream;
    cudaStream_t s = c0->cap_stream;
    cudaGraph_t graph;
    CK(c0, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    pdds_status cap = PDDS_OK;
    auto step = [&](cudaError_t e, const char* what) {
      if (e != cudaSuccess && cap == PDDS_OK) cap = cuda_fail(c0, e, what);
    };
    for (int i = 0; i < count; ++i) {
      pdds_ctx* c = ctxs[i];
      step(cudaMemcpyAsync(G[i]->row_ptr, c->d_row_ptr, (c->geo.n + 1) * 4,
                           cudaMemcpyDeviceToDevice, s), "pattern copy");
      step(cudaMemcpyAsync(G[i]->col, c->d_col, c->geo.nnz * 4, cudaMemcpyDeviceToDevice, s),
           "pattern copy");
      step(cudaMemsetAsync(G[i]->val, 0, c->geo.nnz * 8, s), "memset");
      step(cudaMemsetAsync(b[i], 0, c->geo.n * 8, s), "memset");
    }
    // cleared before the prefixes, which record invalid budgets in it
    step(cudaMemsetAsync(c0->d_scratch, 0, sizeof(pdds::Scratch), s), "memset");
    for (int i = 0; N && i < count; ++i) {
      pdds_ctx* c = ctxs[i];
      if (N[i])
        step(pdds::launch_unit_prefix(N[i], c->geo.n, c0->unit_paths, c->d_unit_prefix,
                                      c->d_path_prefix, &c0->d_scratch->error, s),
             "unit prefix");
    }
    step(pdds::launch_prob_prefix(c0->d_batch, count, c0->d_prob_prefix, s), "prob prefix");
    if (cap == PDDS_OK) {
      const bool timing = c0->timing;
      c0->timing = false;
      // the batch takes the calls between exit checks of its shortest paths
      int calls = 8;
      for (int i = 0; i < count; ++i) calls = std::min(calls, calls_per_check(ctxs[i], dt));
      c0->batch_calls = calls;
      cap = run_paths(c0, probs[0], c0->d_batch, count, dt, seed, kmax, nullptr, s, sb, max_slots,
                      tw, th, c0->coef_id);
      c0->batch_calls = 0;
      c0->timing = timing;
    }
    for (int i = 0; i < count && cap == PDDS_OK; ++i) {
      pdds_ctx* c = ctxs[i];
      step(pdds::launch_finalize(G[i]->row_ptr, G[i]->col, G[i]->val, b[i], N ? N[i] : nullptr,
                                 Nu, c->geo.n, s), "finalize");
    }
    cudaError_t ee = cudaStreamEndCapture(s, &graph);
    if (cap != PDDS_OK) { if (ee == cudaSuccess) cudaGraphDestroy(graph); return cap; }
    CK(c0, ee);
    cudaError_t ie = cudaGraphInstantiate(&c0->graph, graph, 0);
    cudaGraphDestroy(graph);
    CK(c0, ie);
    c0->graph_key = key;
  }
  c0->st = pdds_stats_t{};
  c0->timing_pending = false;
  if (c0->timing) CK(c0, cudaEventRecord(c0->ev0, s));
  CK(c0, cudaGraphLaunch(c0->graph, s));
  if (c0->timing) {
    CK(c0, cudaEventRecord(c0->ev1, s));
    c0->timing_pending = true;
  }
  int launches = 2 + count;
  for (int i = 0; i < count; ++i) launches += (N && N[i]) ? 1 : 0;
  c0->st.kernel_launches = launches;
  return PDDS_OK;
}

pdds_status pdds_assemble_solve_batch_host(pdds_ctx* const* ctxs, int32_t count,
                                           const int64_t* const* N_host, int64_t Nu, double dt,
                                           uint64_t seed, double rtol, int32_t maxit,
                                           int32_t* const* rp_host, int32_t* const* col_host,
                                           double* const* val_host, double* const* b_host,
                                           double* const* u_host, void* stream) {
  if (!ctxs || count < 1 || !ctxs[0])
    return fail(nullptr, PDDS_EINVAL, "assemble_solve_batch_host: need count >= 1 contexts");
  pdds_ctx* c0 = ctxs[0];
  if (!val_host || !b_host || !u_host)
    return fail(c0, PDDS_EINVAL,
                "assemble_solve_batch_host: val, b and u host pointer arrays are required");
  for (int i = 0; i < count; ++i) {
    pdds_ctx* c = ctxs[i];
    if (!c) return fail(c0, PDDS_EINVAL, "assemble_solve_batch_host: NULL context in the list");
    if (!val_host[i] || !b_host[i] || !u_host[i])
      return fail(c0, PDDS_EINVAL, "assemble_solve_batch_host: NULL val, b or u host buffer");
    const int64_t* Nh = N_host ? N_host[i] : nullptr;
    for (int64_t k = 0; Nh && k < c->geo.n; ++k)
      if (Nh[k] < 0 || Nh[k] > 0x7fffffffll)
        return fail(c0, PDDS_EINVAL, "assemble_solve_batch_host: every N_k must be in [0, 2^31)");
  }
  cudaStream_t s = (cudaStream_t)stream;
  // Device buffers: each context's own end-to-end scratch (kept for reuse).
  std::vector<pdds_csr> Gs(count);
  std::vector<pdds_csr*> Gp(count);
  std::vector<double*> bd(count);
  std::vector<const int64_t*> Nd(count, nullptr);
  for (int i = 0; i < count; ++i) {
    pdds_ctx* c = ctxs[i];
    const int64_t n = c->geo.n, nnz = c->geo.nnz;
    if (!c->e_rp) {
      CK(c0, dalloc(&c->e_N, n));
      CK(c0, dalloc(&c->e_rp, n + 1));
      CK(c0, dalloc(&c->e_col, nnz));
      CK(c0, dalloc(&c->e_val, nnz));
      CK(c0, dalloc(&c->e_b, n));
      CK(c0, dalloc(&c->e_u, n));
    }
    if (N_host && N_host[i]) {
      CK(c0, cudaMemcpyAsync(c->e_N, N_host[i], n * 8, cudaMemcpyHostToDevice, s));
      Nd[i] = c->e_N;
    }
    Gs[i] = pdds_csr{n, nnz, c->e_rp, c->e_col, c->e_val};
    Gp[i] = &Gs[i];
    bd[i] = c->e_b;
  }
  if (pdds_status e = pdds_assemble_batch(ctxs, count, N_host ? Nd.data() : nullptr, Nu, dt, seed,
                                          Gp.data(), bd.data(), stream))
    return e;
  pdds_status worst = PDDS_OK;
  int launches = c0->st.kernel_launches;
  for (int i = 0; i < count; ++i) {
    pdds_ctx* c = ctxs[i];
    const int before = c->st.kernel_launches;
    pdds_status se = pdds_solve(c, &Gs[i], c->e_b, c->e_u, rtol, maxit, nullptr, stream);
    if (se != PDDS_OK && se != PDDS_ENOCONV) return c == c0 ? se : fail(c0, se, c->err);
    if (se == PDDS_ENOCONV) worst = PDDS_ENOCONV;
    launches += c->st.kernel_launches - before;
  }
  for (int i = 0; i < count; ++i) {
    pdds_ctx* c = ctxs[i];
    const int64_t n = c->geo.n, nnz = c->geo.nnz;
    if (rp_host && rp_host[i])
      CK(c0, cudaMemcpyAsync(rp_host[i], c->e_rp, (n + 1) * 4, cudaMemcpyDeviceToHost, s));
    if (col_host && col_host[i])
      CK(c0, cudaMemcpyAsync(col_host[i], c->e_col, nnz * 4, cudaMemcpyDeviceToHost, s));
    CK(c0, cudaMemcpyAsync(val_host[i], c->e_val, nnz * 8, cudaMemcpyDeviceToHost, s));
    CK(c0, cudaMemcpyAsync(b_host[i], c->e_b, n * 8, cudaMemcpyDeviceToHost, s));
    CK(c0, cudaMemcpyAsync(u_host[i], c->e_u, n * 8, cudaMemcpyDeviceToHost, s));
  }
  CK(c0, cudaStreamSynchronize(s));
  c0->st.kernel_launches = launches;
  return worst;
}

}  // extern "C"
