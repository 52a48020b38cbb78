// Internal data layout shared by the host setup and the CUDA kernels of the
// PDDSparse assembly library (not part of the public C ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace pdds {

constexpr int kSides = 4;  // patch sides in the order E, N, W, S (Eq. 14)

// One interfacial knot and its patch, as the path kernel needs them (128 B).
// The patch box is stored relative to the knot in FP32 so that paths can be
// integrated in knot-relative coordinates, which keeps FP32 rounding of the
// position ~1e-9 instead of ~6e-8 in absolute coordinates.
struct alignas(16) KnotDesc {
  float xk, yk;            // absolute knot position (FP32, for coefficients)
  float box[4];            // x_lo, x_hi, y_lo, y_hi of the patch, relative to the knot
  int32_t ki, kj;          // lattice coordinates of the knot
  int32_t line[kSides];    // fixed lattice coordinate of each side's grid line
  int32_t a[kSides];       // stencil lattice range [a, b] along the side's line (Eq. 17)
  int32_t b[kSides];
  int32_t off[kSides];     // first accumulator slot of each interface side
  int32_t slot_base;       // offset of this knot's slots in the slot->CSR map
  int32_t nslots;          // slots of this knot (sum over interface sides of b-a+1)
  int32_t dirbits;         // bit o: side o lies on the boundary of Omega (Dirichlet)
  int32_t tile_i0, tile_j0;  // TABLE: table node of the tile's lower-left corner
  float tab_fx, tab_fy;    // TABLE: knot position in tile-local node units
  int32_t pad_;
};
static_assert(sizeof(KnotDesc) == 128, "KnotDesc layout: 32 words, one per lane");

// One problem (a context) as seen by the kernels.
struct ProbDesc {
  int32_t coef_id;
  int32_t n;               // knots
  int32_t LX, LY;          // lattice extents Hx*m, Hy*m
  float params[8];
  float x0, y0, x1, y1;    // Omega
  float dx, dy;            // lattice spacing
  float inv_dx, inv_dy;
  float tab_inv_dx, tab_inv_dy;   // TABLE: table nodes per unit length
  int32_t tag;             // Philox counter word 3
  int32_t pad0_;
  const KnotDesc* knots;
  const int32_t* slot2csr; // CSR value index per slot, -1 for boundary points
  const int64_t* n_per_knot;      // nullable
  int64_t n_paths;                // uniform budget when n_per_knot == nullptr
  const int64_t* knot_unit_prefix; // [n+1] units before knot k (per-knot budgets)
  int64_t units_per_knot;         // uniform budgets
  const int64_t* path_prefix;     // [n+1] records before knot k (records mode)
  double* Gval;
  double* b;
  const CUtensorMap* tmap;        // TABLE: map of the interleaved (sigma, c) table (device)
  int32_t tab_nx, tab_ny;        // TABLE: table nodes
  const int32_t* col;             // CSR column of each value (records mode)
  const double* h_per_knot;       // per-knot steps (extended-exit kernels), or nullptr
  float sigma_max;                // upper bound of s(x) over the closure of Omega
  int32_t rbf_deg;                // RBF stencils: Chebyshev degree of the tables
  const float* rbf_coef;          // RBF stencils (extended kernels), or nullptr: linear
  const int64_t* rbf_off;         // [2][rbf_lmax + 1] table offset per (orientation, length)
  int32_t rbf_lmax;
  int32_t cv_nx;                  // tabulated control variate: nodes per row, or 0
  const float* cv_tab;            // [cv_ny][cv_nx][2] grad u0 spanning Omega, or nullptr
  int32_t cv_ny;
  float cv_inv_dx, cv_inv_dy;     // table nodes per unit length
  int32_t pad1_;
};

// Device-side counters of one launch (zeroed before each assemble).
struct Scratch {
  unsigned long long next_unit;   // global work queue
  unsigned long long steps;
  unsigned long long paths;
  unsigned long long truncated;
  unsigned long long clamped;
  unsigned long long units;
  int32_t error;                  // 0, PDDS_ETIMEOUT or PDDS_EINVAL (missing RBF table, bad budget)
  int32_t pad_;
};

struct PathRecordDev {
  int32_t steps, side_flags, col_a, col_b;
  float w_a, w_b, b_contrib, Y, xi;
  float s_line;  // interface exit: lattice coordinate along the side's line
};
static_assert(sizeof(PathRecordDev) == 40, "record layout of pdds_path_record");

struct KParams {
  ProbDesc prob0;                   // the problem when nprob == 1
  const ProbDesc* probs;            // device array when nprob > 1
  const int64_t* prob_unit_prefix;  // [nprob+1]
  int32_t nprob;
  int32_t exit_batch;
  int32_t calls_per_check;          // Philox calls (two steps each) between a warp's exit checks
  int64_t total_units;
  int64_t unit_paths;
  Scratch* scratch;
  PathRecordDev* records;
  uint32_t key0, key1;
  uint32_t round_keys[20];  // Philox round r: key0 + r W0, key1 + r W1 (rounds 0..9)
  float h, sqh;
  int64_t kmax;
  int32_t max_slots;       // accumulator slots per stage
  int32_t tile_w, tile_h;  // TABLE tile (nodes)
  int32_t stage_bytes;     // bytes per stage in dynamic shared memory
  int32_t mixed;           // records kernels with the extended exit: 1 = mixed GM/EM run
  int32_t pad_;
  PathRecordDev* records_gm;  // mixed run: the Gobet-Menozzi exit of each path
  uint64_t wait_ns;        // bound on any device-side wait
  const void* mlp;         // staged control-variate network (MlpSmem), or nullptr
  int32_t trig_direct;     // the coefficient set's angles are small enough for the hardware
                           // sine without reduction: Omega within [-1, 1]^2 (manufactured),
                           // [-7, 7]^2 (variable sigma) or [-256, 256]^2 (the Poisson
                           // problem of Sec. 5.1)
  int32_t gm;              // extended kernels: 1 = Gobet-Menozzi shift of the sides
  double dt;               // extended kernels: step at which kmax counts
};

// Launchers implemented in the .cu files (host-callable).
// `cv`: 0 none, 1 in-path network, 2 tabulated gradient; `ext` selects the
// extended-exit variants (per-knot steps, Gobet-Menozzi shift, RBF stencils).
cudaError_t launch_path_kernel(int coef_id, bool records, int cv, bool ext, const KParams& kp,
                               int grid, int block, size_t smem, cudaStream_t stream);
cudaError_t path_kernel_occupancy(int coef_id, bool records, int cv, bool ext, int block,
                                  size_t smem, int* ctas_per_sm);
cudaError_t set_path_kernel_smem(int coef_id, bool records, int cv, bool ext, size_t smem);
bool path_kernel_has_cv(int coef_id);
// Control-variate network (pdds_mlp.cu): FP32 theta -> staged image.
size_t mlp_image_bytes();
cudaError_t mlp_stage(const float* theta, void* image, cudaStream_t stream);
// Budgets outside [0, 2^31) count as zero paths and set *err = PDDS_EINVAL.
cudaError_t launch_unit_prefix(const int64_t* n_per_knot, int64_t n, int64_t unit_paths,
                               int64_t* knot_unit_prefix, int64_t* path_prefix, int32_t* err,
                               cudaStream_t stream);
cudaError_t launch_cv_cells(const float* nodes, int nx, int ny, float* cells, cudaStream_t s);
cudaError_t launch_prob_prefix_single(const ProbDesc& D, int64_t* out, cudaStream_t stream);
cudaError_t launch_prob_prefix(const ProbDesc* probs, int nprob, int64_t* out, cudaStream_t stream);
size_t stage_header_bytes();
cudaError_t launch_finalize(const int32_t* row_ptr, const int32_t* col, double* val, double* b,
                            const int64_t* n_per_knot, int64_t n_paths, int64_t n,
                            cudaStream_t stream);

// RBF stencil tables (pdds_rbf.cpp, host): Chebyshev coefficients of the
// cardinal functions of every stencil length, per lattice interval.
struct RbfTables {
  int degree = 0;
  int lmax = 0;
  double max_err = 0;              // coefficient tail bound of the truncation
  double hmax = 0;                 // max |H| seen
  std::vector<float> coef;         // [(t * (degree + 1) + n) * L + j] per table
  std::vector<int64_t> offset;     // [2][lmax + 1], -1 where absent
};
// lengths[o]: stencil lengths of lines along x (o = 0) and y (o = 1);
// c_lat[o]: the shape parameter in units of that orientation's spacing.
bool rbf_build_tables(const std::vector<int> lengths[2], const double c_lat[2], RbfTables& T,
                      std::string& err);
double rbf_shape_for_cond(int m, double cond);  // c (lattice units) with cond(Phi) = cond
double rbf_cond(int m, double c_lat);

// Calibration (pdds_calib.cu): per-knot moments of the mixed GM/EM scores
// from the records of the naive and the Gobet-Menozzi pass, and Eq. 40-41.
// With RBF stencils (D.rbf_coef set) a score's interface part is rebuilt from
// the record's exit side and coordinate with the same tables.
cudaError_t launch_calib_moments(const PathRecordDev* rec_em, const PathRecordDev* rec_gm,
                                 const int64_t* path_prefix, int64_t n_paths, const double* u0,
                                 int64_t n, double* moments, const ProbDesc& D,
                                 cudaStream_t stream);
cudaError_t launch_plan(const double* moments, int64_t n, double eps, double h0, double h0p,
                        int64_t n_job, double* h_out, int64_t* n_out, double* diag,
                        cudaStream_t stream);

// Boundary data g at 4 n points of the boundary of Omega (pdds_path.cu).
cudaError_t launch_boundary_samples(int coef, const double dom[4], const double params[8], int n,
                                    float* xy, float* g, cudaStream_t stream);

// FP64 BiCGSTAB building blocks (pdds_solve.cu).
struct SolveScalars;
cudaError_t bicgstab_device(const int32_t* row_ptr, const int32_t* col, const double* val,
                            const double* b, double* x, int64_t n, double* work,
                            SolveScalars* sc, double rtol, int32_t maxit, int32_t* iters,
                            double* relres, int* converged, int* launches, cudaStream_t stream);
size_t bicgstab_work_doubles(int64_t n);
void set_global_error(const std::string& msg);  // text of pdds_last_error(NULL)
size_t bicgstab_scalars_bytes();
// Why a BiCGSTAB run stopped without converging, from the `converged` output
// of bicgstab_device (negative: a breakdown of the recurrence; 0: maxit).
inline const char* bicgstab_stop_reason(int converged) {
  static const char* why[] = {"", " ((rh,v) = 0)", " (omega = 0)", " ((rh,r) = 0)",
                              " (residual not finite)"};
  return (converged < 0 && -converged <= 4) ? why[-converged] : "";
}

}  // namespace pdds
