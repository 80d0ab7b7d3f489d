// Internal declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <vector>
#include <string>

#ifdef __CUDACC__
#define COFFEE_HD __host__ __device__
#else
#define COFFEE_HD
#endif

namespace coffee {

enum { CELL_TRI = 0, CELL_TET = 1, CELL_PRISM = 2 };
enum { FORM_MASS = 0, FORM_HELMHOLTZ = 1, FORM_ADVDIFF = 2, FORM_BURGERS = 3, FORM_BURGERS_RES = 4 };
// the Burgers residual (an element vector) uses the Burgers Jacobian's reference tensors
inline int table_form(int form) { return form == FORM_BURGERS_RES ? FORM_BURGERS : form; }
inline bool burgers_like(int form) { return form == FORM_BURGERS || form == FORM_BURGERS_RES; }
enum { PREC_FP64 = 0, PREC_TF32 = 1, PREC_TF32X3 = 2, PREC_BF16 = 3, PREC_BF16X3 = 4 };
// Parts of the tensor-core operands per precision (see PrecTraits in tc_common.cuh): the
// reference tensor T and the per-cell factors G are each held as a sum of this many tf32/bf16 values.
COFFEE_HD constexpr int prec_tparts(int prec) {
  return prec == PREC_TF32 ? 1 : prec == PREC_BF16X3 ? 3 : 2;
}
COFFEE_HD constexpr int prec_gparts(int prec) {
  return prec == PREC_TF32X3 ? 2 : prec == PREC_BF16X3 ? 3 : 1;
}

// Device error word bits
enum : unsigned { ERR_INDEX = 1u, ERR_TIMEOUT = 2u, ERR_CAPACITY = 4u };
// Tuning knobs of the tensor-core kernels (from coffee_assemble_args.flags)
enum : unsigned { TUNE_OUTPUT_LANES = 1u, TUNE_TWO_STAGES = 2u, TUNE_SUB64 = 4u, TUNE_SUB32 = 8u, TUNE_SUB128 = 16u,
                  TUNE_CELL_LANES = 32u, TUNE_STAGED_STORE = 128u, TUNE_BURGERS_BLOCKS = 256u,
                  TUNE_BURGERS_FACTORED = 512u };

// ---- host tabulation (tabulate.cpp) ----
int nnodes(int cell, int k);
int npairs(int d);
void pair_index(int d, int p, int& a, int& b);
int quad_degree_for(int form, int k);
int form_K(int form, int k, int cell);
void quadrature_rule(int cell, int degree, std::vector<double>& pts, std::vector<double>& wts);
void lagrange_basis(int cell, int k, int npts, const double* x, double* phi, double* grads);
void reference_tensor(int form, int k, int cell, std::vector<double>& T);

// prisms (tabulate.cpp): rule, basis, per-point reference tensors
int prism_nnodes(int k);
void prism_rule(int k, std::vector<double>& pts, std::vector<double>& wts);
void prism_basis(int k, int npts, const double* x, double* phi, double* grads);
void prism_tensor(int form, int k, std::vector<double>& T, std::vector<double>& pts, std::vector<double>& wts);
void prism_rule_points(int n, std::vector<double>& pts, std::vector<double>& wts);
int prism_burgers_points(int k);
void prism_burgers_table(int k, std::vector<double>& tab, int& Q);

// ---- error reporting (api.cu) ----
int fail(int status, const std::string& msg);
// the allocation-free adjoint's own error word on the current device, read and cleared (noalloc.cu)
int noalloc_error_word(unsigned* w);

// ---- FP64 plain kernel (k_fp64.cu) ----
struct Fp64Params {
  const double* coords;
  const int32_t* c2v;
  const double* coef;
  const int32_t* c2d;
  const double* T;  // [K][N] with N = ns*ns
  void* out;        // double [ncells][ndof][ndof]
  unsigned* err;
  int64_t ncells, nverts, ncoefnodes;
  int64_t ostride;  // entries between consecutive element matrices (element vectors) in out
  int ns, N, ndof;
  double nu;
  int validate;
  const uint32_t* map;  // global assembly: CSR position of every entry (blocked, csr_map_index), else NULL
  int64_t nnz;          // length of the CSR value array (out) when map is set
};
// returns cudaError_t as int
int launch_fp64(int form, int cell, const Fp64Params& p, void* stream);

// ---- FP64 prism kernel (k_prism.cu) ----
struct PrismParams {
  const double* coords;  // [nverts][3]
  const int32_t* c2v;    // [ncells][6]
  const double* coef;    // ADVDIFF: rows (eps, b0, b1, b2) per coefficient node
  const int32_t* c2d;    // ADVDIFF: [ncells][6]
  int64_t ncoefnodes;
  const double* T;       // [Q*KQ][N] per-point tensors, then points [Q][3], then weights [Q]
  void* out;             // double [ncells][N], or the CSR values when map is set
  unsigned* err;
  int64_t ncells, nverts;
  int Q, N;
  int validate;
  const uint32_t* map;   // global assembly (blocked entry map), else NULL
  int64_t nnz;
  double nu;             // Burgers viscosity
};
int launch_prism(int form, const PrismParams& p, int num_sms, void* stream);
// vector Burgers on prisms, FP64 (k_prism_burgers.cu): the Jacobian (FORM_BURGERS) or the residual
// (FORM_BURGERS_RES); p.T holds prism_burgers_table, p.N the nodes n of one component, p.Q points
int launch_prism_burgers(int form, int degree, const PrismParams& p, int num_sms, void* stream);
// tensor-core prisms (k_prism_tc.cu): K-chunked streamed contraction, MASS/HELMHOLTZ/ADVDIFF P1-P4
struct TcParams;
struct TcTable;
int prism_tc_supported(int form, int degree, int precision);

// ---- adjoint (k_bwd.cu) ----
struct BwdParams {
  const double* coords;
  const int32_t* c2v;
  const double* coef;
  const int32_t* c2d;
  const double* T;       // FP64 reference tensors [K][N]
  const void* dout;      // [ncells][N], double or float
  int dout_fp32;
  double* d_coords;      // accumulated (atomic mode)
  double* d_coef;        // accumulated (atomic mode), may be NULL
  double* local;         // deterministic mode: per-cell contributions [ncells][nl], else NULL
  unsigned* err;
  int64_t ncells, nverts, ncoefnodes;
  int N;
  int validate;
};
int bwd_local_len(int form, int cell);
int launch_backward(int form, int cell, const BwdParams& p, void* stream);
int launch_ordered_sum(const int32_t* idx, int64_t ncells, int width, int64_t nnodes, const double* local,
                       int nl, int base, int comps, double* grad, int grad_stride, int grad_off,
                       int32_t* cnt, int32_t* cursor, int64_t* off, int64_t* slots, unsigned* err,
                       void* stream);

// ---- tcgen05 tensor-core contraction (k_tc.cu) ----
// Operand image of the reference tensor for the tensor cores: for each M-tile of
// 128 output rows, the tparts parts of T^T (the first the round-to-nearest of T, each next
// one of what the previous left), each 128 rows x kbytes bytes in the canonical no-swizzle
// K-major core-matrix layout.
struct TcTable {
  const uint8_t* image;  // device
  int mtiles;            // ceil(N / 128) (per block for Burgers)
  int kbytes;            // bytes per operand row (multiple of 32)
  int kelems;            // padded K (elements)
  int K;                 // true K
  int tparts;            // parts of T held per M-tile (1, 2 or 3; 1 when aexact)
  int ksteps_off;        // Burgers: K-steps of the off-diagonal component blocks
  int64_t tile_bytes;    // bytes of one part of one M-tile = 128 * kbytes
  int aexact;            // 1: every A column is an integer vector times a scale, so A is held
                         // exactly in one part and the scales (float [kelems]) follow the tiles
  int64_t scale_off;     // byte offset of those scales in the image
  int64_t aux_off;       // Burgers Jacobian: offset of the factored-form image (0: none)
  int aux_vparts, aux_cparts;  // its parts of the T1 and of the T2|T3 operands
};

struct TcParams {
  const double* coords;
  const float* xs;       // optional: every coordinate as (hi, lo) floats, [nverts][d][2]
  const int32_t* c2v;
  const double* coef;
  const float* cf;       // optional: coef rounded to float, same layout
  const int32_t* c2d;
  const uint8_t* image;  // TcTable image
  float* out;
  unsigned* err;
  int64_t ncells, nverts, ncoefnodes;
  int64_t ostride;       // entries between consecutive element matrices in out (N when contiguous)
  int ns, N;             // outputs per cell
  int mtiles, kbytes, tparts;  // tparts: TcTable::tparts
  int ksteps_off;        // Burgers: K-steps of the off-diagonal component blocks
  unsigned tune;         // TUNE_* knobs
  int subw;              // cells per TMEM accumulator (outputs-on-lanes orientation)
  int stage_cells;       // staged epilogue: rows per bulk copy (0: direct stores)
  int stage_bufs;        // staged epilogue: buffers of stage_cells rows (2 to 4)
  int precision;
  int validate;
  double nu;
  const uint32_t* map;   // global assembly: CSR position of every entry (blocked, csr_map_index); out = CSR values
  int64_t nnz;           // length of the CSR value array when map is set
  int nkc;               // prisms: K-chunks of the streamed contraction
  int aexact;            // TcTable::aexact
  int64_t scale_off;     // TcTable::scale_off
  int64_t aux_off;       // TcTable::aux_off
  int aux_vparts, aux_cparts;
};
int tc_supported(int form, int degree, int cell, int precision);
// staged epilogue (k_tc_staged.cu): its sub-tile width, rows per bulk copy and the bytes of one
// buffer of those rows for p (0 when p cannot take it), and the launch
int staged_plan(const TcParams& p, int& subw, int& cells, int& buf_bytes);
int launch_tc_staged(int form, int cell, const TcParams& q, int num_sms, void* stream, int nst, int smem);
int launch_tc(int form, int cell, const TcParams& p, int num_sms, void* stream, std::string& why);
// T [K][N] (FP64) of the tensor-core contraction: the stiffness tensors in the edge basis
void tc_reference_tensor(int form, int degree, int cell, std::vector<double>& T);
// CUDA-core kernel for small element matrices (k_simt.cu): MASS, HELMHOLTZ and ADVDIFF on
// triangles P1-P3 and tetrahedra P1-P2, FP32; simt_default: where it is the default path
int simt_supported(int form, int degree, int cell);
int simt_default(int form, int degree, int cell);
int launch_simt(int form, int degree, int cell, const TcParams& p, int num_sms, void* stream, std::string& why);
// the CUDA-core share of a mixed batch: groups whose 32-cell warp tiles are numbered from tile0
struct SimtGroup {
  TcParams p;
  int64_t tile0;
  int kind;  // simt_kind(form, degree, cell)
};
int simt_kind(int form, int degree, int cell);
int simt_upload(int form, int degree, int cell);
int launch_simt_batch(const SimtGroup* groups, int ngroups, int64_t ntiles, int num_sms, void* stream);
// Burgers-Jacobian tensor-core kernel (k_tc_burgers.cu)
int burgers_tc_supported(int degree, int cell, int precision);
void build_burgers_image(int degree, int cell, int prec, bool exact_ok, std::vector<uint8_t>& img, TcTable& meta);
int launch_burgers_tc(int cell, const TcParams& p, int num_sms, void* stream, std::string& why);
// Burgers Jacobian with both operands streamed in K-chunks (k_tc_burgers_stream.cu): tetrahedra
// P3-P4 and triangles P4, where the resident-operand kernel does not fit
int burgers_stream_supported(int degree, int cell, int precision);
void build_burgers_stream_image(int degree, int cell, int prec, std::vector<uint8_t>& img, TcTable& meta);
int launch_burgers_stream_tc(int cell, int degree, const TcParams& p, int num_sms, void* stream, std::string& why);
// Burgers-residual (element vector) tensor-core kernel (k_tc_burgers_res.cu)
int burgers_res_tc_supported(int degree, int cell, int precision);
void build_burgers_res_image(int degree, int cell, int prec, std::vector<uint8_t>& img, TcTable& meta);
// integer form of an operand column (k_tc_burgers.cu): x = n * scale with n exact in the type
bool integer_column(const std::vector<double>& x, bool tf32, double& scale, std::vector<double>& n);
// Burgers Jacobian in the factored form (k_tc_burgers_fact.cu): element matrices of at most 128
// entries per component block; the image is appended to the block kernel's (TcTable::aux_off)
int burgers_fact_supported(int degree, int cell, int precision);
int burgers_fact_default(int degree, int cell);
void build_burgers_fact_image(int degree, int cell, int prec, std::vector<uint8_t>& img, int& vparts, int& cparts);
int launch_burgers_fact_tc(int cell, const TcParams& p, int num_sms, void* stream, std::string& why);
int launch_burgers_res_tc(int cell, const TcParams& p, int num_sms, void* stream, std::string& why);
// ---- mixed-batch persistent kernel (k_batch.cu) ----
struct BatchGroup {
  TcParams p;      // the group's inputs, output, table image, N, mtiles, kbytes
  int64_t item0;   // first work item (128-cell tile) of the group in the work list
  int form, cell, degree;
  int lanes;       // 1: cells on the TMEM lanes (element matrices of at most 32 entries)
};
struct BatchLaunch {
  const BatchGroup* groups;  // device
  int ngroups;
  const int64_t* ranges;     // device [grid+1]: work items of CTA b are [ranges[b], ranges[b+1])
  int grid, smem, nstages, kbytes_max, precision;
  unsigned* err;
};
int batch_smem(int kbytes_max, int precision, int* nstages);
// diagnostic bounded wait that runs out (k_peaks.cu)
int launch_diag_wait(unsigned* err, void* stream);
int batch_prepare(int precision, int smem);
int batch_launch(const BatchLaunch& L, void* stream);
int stream_one_supported(int form, int kbytes, int precision);
int launch_stream_one(const BatchGroup& g, int num_sms, void* stream);

// ---- global assembly (k_csr.cu, k_tc_csr.cu) ----
constexpr int CSR_ROW_CAP = 4096;  // entries of one row before deduplication (sum of nloc over incident cells)
// Entry map of global assembly, blocked as the fused epilogue consumes it: cells in groups of 32
// (padded), entries (npad = n2 rounded up to 4) in groups of 32; block (cb, ob) = [32 cells][width]
// at offset 32*(cb*npad + 32*ob).
inline int64_t csr_map_len(int64_t ncells, int nloc) {
  return (ncells + 31) / 32 * 32 * (int64_t)((nloc * nloc + 3) & ~3);
}
COFFEE_HD inline int64_t csr_map_index(int64_t e, int idx, int npad) {
  const int ob = idx >> 5, bw = npad - ob * 32 < 32 ? npad - ob * 32 : 32;
  return 32 * ((e >> 5) * (int64_t)npad + 32 * ob) + (e & 31) * bw + (idx & 31);
}
size_t sparsity_scratch_bytes(int64_t ncells, int nloc, int64_t nrows);
int launch_sparsity(const int32_t* l2g, int64_t ncells, int nloc, int64_t nrows, int64_t* rowptr, int32_t* colidx,
                    uint8_t* ws, unsigned** flag, int num_sms, void* stream);
int launch_csr_map(const int32_t* l2g, int64_t ncells, int nloc, const int64_t* rowptr, const int32_t* colidx,
                   int64_t nrows, uint32_t* map, unsigned* err, int num_sms, void* stream);
int tc_csr_supported(int form, int degree, int cell, int precision);
void build_prism_tc_image(int form, int degree, int prec, std::vector<uint8_t>& img, TcTable& meta);
int launch_prism_tc(int form, int degree, const TcParams& p, int num_sms, void* stream, std::string& why);
int launch_tc_csr(int form, int cell, const TcParams& p, int num_sms, void* stream, std::string& why);

// Build the operand image on the host
void build_tc_image(int form, int degree, int cell, int precision, std::vector<uint8_t>& img,
                    TcTable& meta);

}  // namespace coffee
