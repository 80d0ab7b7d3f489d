// C-ABI entry points of libcoffee.so (declared in include/coffee.h): argument
// validation, the per-device cache of reference tensors, and kernel dispatch.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>
#include "../../include/coffee.h"
#include "../../include/coffee_diag.h"
#include "coffee_internal.h"
#include "tc_common.cuh"

namespace coffee {

// The two per-node conversion kernels below (coordinates, coefficients) move a few MB each. They
// convert by integer operations: FP64 instructions, conversions included, issue at 1/16 of a
// warp per SM cycle on this GPU, which made both kernels FP64-bound (ncu: SM 64% busy, DRAM 10%).
// The FP64 forms run out of line (a call, so the compiler cannot if-convert them into every
// thread's path) for the values the integer forms do not cover. With one 16-byte load in flight
// per thread a full GPU holds about 5 MB of loads at once, so each thread issues UNROLL
// independent 16-byte loads before it converts and stores any of them.
constexpr int UNROLL = 4;

__device__ __noinline__ float2 split_pair_f64(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

// x as a float pair (hi, lo) with hi + lo = x to 2^-48 of |x| (lo a normal float:
// 2^-100 <= |x| < 2^127). In the range split_exact takes (|x| in [2^-70, 2^100)), hi is x
// truncated to 24 significant bits and lo the rest; outside it hi = (float)x, lo = (float)(x - hi).
__device__ __forceinline__ float2 split_pair(double v) {
  float hi, lo;
  if (!tc::split_exact(v, hi, lo)) return split_pair_f64(v);
  return make_float2(hi, lo);
}

__device__ __noinline__ float f32_of_f64(double v) { return (float)v; }

// The float nearest to v, ties to even (IEEE 754 round to nearest): where the result is a normal
// float (biased exponent e of v in [897, 1150], |v| in [2^-126, 2^128)) the float's exponent is
// e - 896 and its 23 fraction bits are v's top 23; the 29 bits below decide: above half an ulp,
// or exactly half with an odd result, add one ulp (a carry moves into the exponent, up to
// infinity past the largest float, as rounding to nearest gives). Zero, results below 2^-126,
// infinities and NaN take the conversion instruction.
__device__ __forceinline__ float f32_rn(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const uint32_t h = (uint32_t)(b >> 32), l = (uint32_t)b;
  const uint32_t ef = h & 0x7FF00000u;
  if (ef - (897u << 20) > ((1150u - 897u) << 20)) return f32_of_f64(v);
  const uint32_t f = __funnelshift_l(l, (h & 0x7FFFFFFFu) - (896u << 20), 3);
  const uint32_t rem = l & 0x1FFFFFFFu;
  const uint32_t up = (uint32_t)(rem > 0x10000000u) | ((uint32_t)(rem == 0x10000000u) & f);
  return __uint_as_float(((f + (up & 1u))) | (h & 0x80000000u));
}

// every coordinate as its (hi, lo) pair: the coords_split input
__global__ void k_split_coords(const double* __restrict__ x, int64_t n, float2* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool vec = ((reinterpret_cast<uintptr_t>(x) & 15u) == 0) && ((reinterpret_cast<uintptr_t>(out) & 15u) == 0);
  if (vec) {  // pairs of coordinates: 16 bytes in, 16 out
    const int64_t n2 = n / 2;
    const double2* x2 = reinterpret_cast<const double2*>(x);
    float4* o4 = reinterpret_cast<float4*>(out);
    for (int64_t b = i0; b < n2; b += UNROLL * stride) {
      double2 v[UNROLL];
#pragma unroll
      for (int j = 0; j < UNROLL; ++j) {
        const int64_t i = b + j * stride;
        v[j] = i < n2 ? __ldcs(x2 + i) : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int j = 0; j < UNROLL; ++j) {
        const int64_t i = b + j * stride;
        if (i < n2) {
          const float2 a = split_pair(v[j].x), c = split_pair(v[j].y);
          o4[i] = make_float4(a.x, a.y, c.x, c.y);
        }
      }
    }
    if (i0 == 0 && (n & 1)) out[n - 1] = split_pair(x[n - 1]);
  } else {
    for (int64_t i = i0; i < n; i += stride) out[i] = split_pair(x[i]);
  }
}

// every coefficient rounded to the nearest float: the coef_f32 input
__global__ void k_round_coef(const double* __restrict__ x, int64_t n, float* __restrict__ out) {
  const int64_t n2 = n / 2;  // pairs, when both pointers allow 16- and 8-byte accesses
  const bool vec = ((reinterpret_cast<uintptr_t>(x) & 15u) == 0) && ((reinterpret_cast<uintptr_t>(out) & 7u) == 0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (vec) {
    for (int64_t b = i0; b < n2; b += UNROLL * stride) {
      double2 v[UNROLL];
#pragma unroll
      for (int j = 0; j < UNROLL; ++j) {
        const int64_t i = b + j * stride;
        v[j] = i < n2 ? __ldcs(reinterpret_cast<const double2*>(x) + i) : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int j = 0; j < UNROLL; ++j) {
        const int64_t i = b + j * stride;
        if (i < n2) reinterpret_cast<float2*>(out)[i] = make_float2(f32_rn(v[j].x), f32_rn(v[j].y));
      }
    }
    if (i0 == 0 && (n & 1)) out[n - 1] = f32_rn(x[n - 1]);
  } else {
    for (int64_t i = i0; i < n; i += stride) out[i] = f32_rn(x[i]);
  }
}

static thread_local std::string g_last_error;

int fail(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}

static int cuda_fail(cudaError_t e, const char* where) {
  return fail(COFFEE_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

namespace {

struct TcEntry {
  uint8_t* image = nullptr;
  TcTable meta{};
};

struct DeviceCache {
  unsigned* err = nullptr;
  int num_sms = 0;
  std::map<std::tuple<int, int, int>, double*> fp64;    // (form, degree, cell)
  std::map<std::tuple<int, int, int, int>, TcEntry> tc;  // + precision
};

std::mutex g_mu;
std::map<int, DeviceCache> g_cache;

int device_cache(DeviceCache** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  DeviceCache& c = g_cache[dev];
  if (!c.err) {
    e = cudaMalloc(&c.err, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(error word)");
    e = cudaMemset(c.err, 0, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(error word)");
    e = cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  }
  *out = &c;
  return COFFEE_OK;
}

int fp64_table(DeviceCache& c, int form, int degree, int cell, const double** T) {
  form = table_form(form);
  auto key = std::make_tuple(form, degree, cell);
  auto it = c.fp64.find(key);
  if (it != c.fp64.end()) {
    *T = it->second;
    return COFFEE_OK;
  }
  std::vector<double> h;
  if (cell == CELL_PRISM && form == FORM_BURGERS) {
    // the basis at the Burgers rule's points, then the points and weights
    int Q = 0;
    prism_burgers_table(degree, h, Q);
  } else if (cell == CELL_PRISM) {
    // per-point tensors, then the rule's points and weights (read by the prism kernel)
    std::vector<double> pts, wts;
    prism_tensor(form, degree, h, pts, wts);
    h.insert(h.end(), pts.begin(), pts.end());
    h.insert(h.end(), wts.begin(), wts.end());
  } else {
    reference_tensor(form, degree, cell, h);
  }
  double* d = nullptr;
  cudaError_t e = cudaMalloc(&d, h.size() * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(reference tensor)");
  e = cudaMemcpy(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_fail(e, "cudaMemcpy(reference tensor)");
  }
  c.fp64[key] = d;
  *T = d;
  return COFFEE_OK;
}

int tc_table(DeviceCache& c, int form, int degree, int cell, int prec, TcTable* meta) {
  auto key = std::make_tuple(form, degree, cell, prec);
  auto it = c.tc.find(key);
  if (it == c.tc.end()) {
    std::vector<uint8_t> img;
    TcEntry ent;
    build_tc_image(form, degree, cell, prec, img, ent.meta);
    cudaError_t e = cudaMalloc(&ent.image, img.size());
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(tensor-core table)");
    e = cudaMemcpy(ent.image, img.data(), img.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(ent.image);
      return cuda_fail(e, "cudaMemcpy(tensor-core table)");
    }
    ent.meta.image = ent.image;
    it = c.tc.emplace(key, ent).first;
  }
  *meta = it->second.meta;
  return COFFEE_OK;
}

bool valid_fdc(int form, int degree, int cell) {
  return form >= FORM_MASS && form <= FORM_BURGERS_RES && degree >= 1 && degree <= 4 &&
         (cell == CELL_TRI || cell == CELL_TET || cell == CELL_PRISM);
}

int check_args(const coffee_assemble_args* a) {
  if (!a) return fail(COFFEE_ERR_INVALID_ARG, "args is NULL");
  if (!valid_fdc(a->form, a->degree, a->cell))
    return fail(COFFEE_ERR_INVALID_ARG, "form/degree/cell out of range (degree 1..4, tri/tet/prism)");
  if (a->precision < PREC_FP64 || a->precision > PREC_BF16X3)
    return fail(COFFEE_ERR_INVALID_ARG, "precision out of range");
  if (a->ncells < 0) return fail(COFFEE_ERR_INVALID_ARG, "ncells < 0");
  if (a->ncells == 0) return COFFEE_OK;
  if (!a->coords || !a->cell2vert || !a->out)
    return fail(COFFEE_ERR_INVALID_ARG, "coords, cell2vert and out must be non-NULL");
  if ((a->flags & COFFEE_FLAG_VALIDATE) && a->nverts <= 0)
    return fail(COFFEE_ERR_INVALID_ARG, "validation needs nverts > 0");
  if (a->form == FORM_ADVDIFF || burgers_like(a->form)) {
    if (!a->coef || !a->cell2dof)
      return fail(COFFEE_ERR_INVALID_ARG, "this form needs coef and cell2dof");
    if (a->ncoefnodes <= 0) return fail(COFFEE_ERR_INVALID_ARG, "ncoefnodes must be > 0");
  }
  if (a->ncells > (int64_t)INT32_MAX * 128)
    return fail(COFFEE_ERR_INVALID_ARG, "ncells too large");
  if (a->out_stride != 0) {
    const int nd = coffee_ndof(a->form, a->degree, a->cell);
    const int64_t N = a->form == FORM_BURGERS_RES ? nd : (int64_t)nd * nd;
    if (a->out_stride != N) {
      if (a->out_stride < N) return fail(COFFEE_ERR_INVALID_ARG, "out_stride is below the element matrix size");
      if (!(a->form == FORM_MASS || a->form == FORM_HELMHOLTZ || a->form == FORM_ADVDIFF) || a->cell == CELL_PRISM)
        return fail(COFFEE_ERR_INVALID_ARG,
                    "out_stride: padded rows for MASS, HELMHOLTZ and ADVDIFF on triangles and tetrahedra only");
    }
  }
  return COFFEE_OK;
}

// Local assembly (map == NULL: element matrices to a->out) or fused global assembly
// (map != NULL: entries added into the CSR values a->out at map[cell][entry]).
int assemble_impl(const coffee_assemble_args* a, const uint32_t* map, int64_t nnz, coffee_stream_t stream) {
  int rc = check_args(a);
  if (rc != COFFEE_OK || a->ncells == 0) return rc;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceCache* c = nullptr;
  if ((rc = device_cache(&c)) != COFFEE_OK) return rc;
  const int d = a->cell == CELL_TRI ? 2 : 3;
  const bool validate = (a->flags & COFFEE_FLAG_VALIDATE) != 0;
  if (a->cell == CELL_PRISM && a->precision != PREC_FP64) {
    if (!prism_tc_supported(a->form, a->degree, a->precision))
      return fail(COFFEE_ERR_UNSUPPORTED, "tensor-core prisms: MASS, HELMHOLTZ and ADVDIFF, P1-P4");
    TcTable meta{};
    if ((rc = tc_table(*c, a->form, a->degree, a->cell, a->precision, &meta)) != COFFEE_OK) return rc;
    TcParams p{};
    p.coords = a->coords;
    p.c2v = a->cell2vert;
    p.coef = a->coef;
    p.cf = a->coef_f32;
    p.c2d = a->cell2dof;
    p.ncoefnodes = a->ncoefnodes;
    p.image = meta.image;
    p.out = static_cast<float*>(a->out);
    p.err = c->err;
    p.ncells = a->ncells;
    p.nverts = a->nverts;
    p.precision = a->precision;
    p.validate = validate ? 1 : 0;
    p.map = map;
    p.nnz = nnz;
    std::string why;
    cudaError_t e = (cudaError_t)launch_prism_tc(a->form, a->degree, p, c->num_sms, stream, why);
    if (e != cudaSuccess) return cuda_fail(e, ("launch(assemble_prism_tc) " + why).c_str());
    return COFFEE_OK;
  }
  if (a->cell == CELL_PRISM && burgers_like(a->form)) {
    if (map && a->form == FORM_BURGERS_RES) return fail(COFFEE_ERR_UNSUPPORTED, "global assembly of element vectors");
    const double* T = nullptr;
    if ((rc = fp64_table(*c, a->form, a->degree, a->cell, &T)) != COFFEE_OK) return rc;
    const int pb = prism_burgers_points(a->degree);
    PrismParams p{};
    p.coords = a->coords;
    p.c2v = a->cell2vert;
    p.coef = a->coef;
    p.c2d = a->cell2dof;
    p.ncoefnodes = a->ncoefnodes;
    p.T = T;
    p.out = a->out;
    p.err = c->err;
    p.ncells = a->ncells;
    p.nverts = a->nverts;
    p.Q = pb * pb * pb;
    p.N = prism_nnodes(a->degree);
    p.validate = validate ? 1 : 0;
    p.nu = a->nu;
    p.map = map;
    p.nnz = nnz;
    cudaError_t e = (cudaError_t)launch_prism_burgers(a->form, a->degree, p, c->num_sms, stream);
    if (e != cudaSuccess) return cuda_fail(e, "launch(prism_burgers)");
    return COFFEE_OK;
  }
  if (a->cell == CELL_PRISM) {
    if (!(a->form == FORM_MASS || a->form == FORM_HELMHOLTZ || a->form == FORM_ADVDIFF))
      return fail(COFFEE_ERR_UNSUPPORTED, "prisms: MASS, HELMHOLTZ and ADVDIFF");
    const double* T = nullptr;
    if ((rc = fp64_table(*c, a->form, a->degree, a->cell, &T)) != COFFEE_OK) return rc;
    const int n = prism_nnodes(a->degree);
    PrismParams p{};
    p.coords = a->coords;
    p.c2v = a->cell2vert;
    p.coef = a->coef;
    p.c2d = a->cell2dof;
    p.ncoefnodes = a->ncoefnodes;
    p.T = T;
    p.out = a->out;
    p.err = c->err;
    p.ncells = a->ncells;
    p.nverts = a->nverts;
    p.Q = (a->degree + 2) * (a->degree + 2) * (a->degree + 2);
    p.N = n * n;
    p.validate = validate ? 1 : 0;
    p.map = map;
    p.nnz = nnz;
    cudaError_t e = (cudaError_t)launch_prism(a->form, p, c->num_sms, stream);
    if (e != cudaSuccess) return cuda_fail(e, "launch(assemble_prism)");
    return COFFEE_OK;
  }
  const int ns = nnodes(a->cell, a->degree);
  const int ndof = burgers_like(a->form) ? d * ns : ns;
  if (a->precision == PREC_FP64) {
    const double* T = nullptr;
    if ((rc = fp64_table(*c, a->form, a->degree, a->cell, &T)) != COFFEE_OK) return rc;
    Fp64Params p{};
    p.coords = a->coords;
    p.c2v = a->cell2vert;
    p.coef = a->coef;
    p.c2d = a->cell2dof;
    p.T = T;
    p.out = a->out;
    p.err = c->err;
    p.ncells = a->ncells;
    p.nverts = a->nverts;
    p.ncoefnodes = a->ncoefnodes;
    p.ns = ns;
    p.N = ns * ns;
    p.ndof = ndof;
    p.ostride = a->out_stride ? a->out_stride : (a->form == FORM_BURGERS_RES ? ndof : (int64_t)ndof * ndof);
    p.nu = a->nu;
    p.validate = validate ? 1 : 0;
    p.map = map;
    p.nnz = nnz;
    cudaError_t e = (cudaError_t)launch_fp64(a->form, a->cell, p, stream);
    if (e != cudaSuccess) return cuda_fail(e, "launch(assemble_fp64)");
    return COFFEE_OK;
  }
  if (map ? !tc_csr_supported(a->form, a->degree, a->cell, a->precision)
          : !tc_supported(a->form, a->degree, a->cell, a->precision))
    return fail(COFFEE_ERR_UNSUPPORTED, map ? "no fused tensor-core global assembly for this form/degree/cell/precision"
                                              : "no tensor-core kernel for this form/degree/cell/precision");
  TcTable meta{};
  if ((rc = tc_table(*c, a->form, a->degree, a->cell, a->precision, &meta)) != COFFEE_OK) return rc;
  TcParams p{};
  p.coords = a->coords;
  p.c2v = a->cell2vert;
  p.coef = a->coef;
  p.c2d = a->cell2dof;
  p.image = meta.image;
  p.xs = a->coords_split;
  p.cf = a->coef_f32;
  p.out = static_cast<float*>(a->out);
  p.err = c->err;
  p.ncells = a->ncells;
  p.nverts = a->nverts;
  p.ncoefnodes = a->ncoefnodes;
  p.ns = ns;
  p.N = ndof * ndof;
  p.ostride = a->out_stride ? a->out_stride : (a->form == FORM_BURGERS_RES ? ndof : (int64_t)ndof * ndof);
  p.mtiles = meta.mtiles;
  p.kbytes = meta.kbytes;
  p.tparts = meta.tparts;
  p.ksteps_off = meta.ksteps_off;
  p.aexact = meta.aexact;
  p.scale_off = meta.scale_off;
  p.aux_off = meta.aux_off;
  p.aux_vparts = meta.aux_vparts;
  p.aux_cparts = meta.aux_cparts;
  p.tune = ((a->flags & COFFEE_FLAG_OUTPUT_LANES) ? TUNE_OUTPUT_LANES : 0u) |
           ((a->flags & COFFEE_FLAG_TWO_STAGES) ? TUNE_TWO_STAGES : 0u) |
           ((a->flags & COFFEE_FLAG_SUBTILE_64) ? TUNE_SUB64 : 0u) |
           ((a->flags & COFFEE_FLAG_SUBTILE_32) ? TUNE_SUB32 : 0u) |
           ((a->flags & COFFEE_FLAG_SUBTILE_128) ? TUNE_SUB128 : 0u) |
           ((a->flags & COFFEE_FLAG_CELL_LANES) ? TUNE_CELL_LANES : 0u) |
           ((a->flags & COFFEE_FLAG_STAGED_STORE) ? TUNE_STAGED_STORE : 0u) |
           ((a->flags & COFFEE_FLAG_BURGERS_BLOCKS) ? TUNE_BURGERS_BLOCKS : 0u) |
           ((a->flags & COFFEE_FLAG_BURGERS_FACTORED) ? TUNE_BURGERS_FACTORED : 0u);
  p.precision = a->precision;
  p.validate = validate ? 1 : 0;
  p.nu = a->nu;
  p.map = map;
  p.nnz = nnz;
  std::string why;
  const bool simt = !map && simt_supported(a->form, a->degree, a->cell) && !(a->flags & COFFEE_FLAG_TENSOR_CORES) &&
                    ((a->flags & COFFEE_FLAG_CUDA_CORES) || simt_default(a->form, a->degree, a->cell));
  if (simt) {
    cudaError_t e = (cudaError_t)launch_simt(a->form, a->degree, a->cell, p, c->num_sms, stream, why);
    if (e != cudaSuccess) return cuda_fail(e, ("launch(assemble_simt) " + why).c_str());
    return COFFEE_OK;
  }
  cudaError_t e = map ? (cudaError_t)launch_tc_csr(a->form, a->cell, p, c->num_sms, stream, why)
                      : (cudaError_t)launch_tc(a->form, a->cell, p, c->num_sms, stream, why);
  if (e != cudaSuccess)
    return cuda_fail(e, ((map ? "launch(assemble_tc_csr) " : "launch(assemble_tc) ") + why).c_str());
  return COFFEE_OK;
}

}  // namespace
}  // namespace coffee

using namespace coffee;

extern "C" {

int coffee_ndof(int form, int degree, int cell) {
  if (!(form >= 0 && form <= 4 && degree >= 1 && degree <= 6 && (cell == 0 || cell == 1 || cell == 2)))
    return fail(COFFEE_ERR_INVALID_ARG, "form/degree/cell out of range");
  if (cell == CELL_PRISM) return burgers_like(form) ? 3 * prism_nnodes(degree) : prism_nnodes(degree);
  int ns = nnodes(cell, degree);
  return burgers_like(form) ? (cell == CELL_TRI ? 2 : 3) * ns : ns;
}

int coffee_tabulate(int cell, int degree, int quad_degree, int* nq, int* ndof, double* points,
                    double* weights, double* basis, double* grads) {
  if (!(cell == 0 || cell == 1) || degree < 1 || degree > 6 || quad_degree < 0 || quad_degree > 30)
    return fail(COFFEE_ERR_INVALID_ARG, "cell/degree/quad_degree out of range");
  std::vector<double> pts, wts;
  quadrature_rule(cell, quad_degree, pts, wts);
  const int n = (int)wts.size(), nd = nnodes(cell, degree), d = cell == 0 ? 2 : 3;
  if (nq) *nq = n;
  if (ndof) *ndof = nd;
  if (points) std::memcpy(points, pts.data(), pts.size() * sizeof(double));
  if (weights) std::memcpy(weights, wts.data(), wts.size() * sizeof(double));
  if (basis || grads) lagrange_basis(cell, degree, n, pts.data(), basis, grads);
  (void)d;
  return COFFEE_OK;
}

int coffee_reference_tensor(int form, int degree, int cell, int* K, int* N, double* T) {
  if (!valid_fdc(form, degree, cell)) return fail(COFFEE_ERR_INVALID_ARG, "form/degree/cell out of range");
  if (cell == CELL_PRISM)
    return fail(COFFEE_ERR_UNSUPPORTED, "prisms are not affine: their Jacobian varies over the cell, so no "
                                        "reference tensor exists (the prism kernels contract per quadrature point)");
  form = table_form(form);
  const int ns = nnodes(cell, degree);
  if (K) *K = form_K(form, degree, cell);
  if (N) *N = ns * ns;
  if (T) {
    std::vector<double> h;
    reference_tensor(form, degree, cell, h);
    std::memcpy(T, h.data(), h.size() * sizeof(double));
  }
  return COFFEE_OK;
}

int coffee_supported(int form, int degree, int cell, int precision) {
  if (!valid_fdc(form, degree, cell) || precision < PREC_FP64 || precision > PREC_BF16X3) return 0;
  if (cell == CELL_PRISM)
    return ((form == FORM_MASS || form == FORM_HELMHOLTZ || form == FORM_ADVDIFF) &&
            (precision == PREC_FP64 || prism_tc_supported(form, degree, precision))) ||
           (burgers_like(form) && precision == PREC_FP64);
  if (precision == PREC_FP64) return 1;
  return tc_supported(form, degree, cell, precision);
}

int coffee_assemble_path(int form, int degree, int cell, int precision, unsigned flags) {
  if (!coffee_supported(form, degree, cell, precision))
    return fail(COFFEE_ERR_UNSUPPORTED, "no kernel for this form/degree/cell/precision");
  if (precision == PREC_FP64) return 0;
  const bool simt = simt_supported(form, degree, cell) && !(flags & COFFEE_FLAG_TENSOR_CORES) &&
                    ((flags & COFFEE_FLAG_CUDA_CORES) || simt_default(form, degree, cell));
  return simt ? 2 : 1;
}

int coffee_round_coef(const double* coef, int64_t n, float* out, coffee_stream_t stream) {
  if (n < 0) return fail(COFFEE_ERR_INVALID_ARG, "round_coef: n < 0");
  if (n == 0) return COFFEE_OK;
  if (!coef || !out) return fail(COFFEE_ERR_INVALID_ARG, "round_coef: coef and out must be non-NULL");
  DeviceCache* c = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    int rc = device_cache(&c);
    if (rc != COFFEE_OK) return rc;
  }
  const int64_t blocks = std::min<int64_t>((n / 2 + 255) / 256 + 1, (int64_t)c->num_sms * 8);
  k_round_coef<<<(unsigned)blocks, 256, 0, stream>>>(coef, n, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "launch(round_coef)");
  return COFFEE_OK;
}

int coffee_split_coords(const double* coords, int64_t n, float* split, coffee_stream_t stream) {
  if (n < 0) return fail(COFFEE_ERR_INVALID_ARG, "split_coords: n < 0");
  if (n == 0) return COFFEE_OK;
  if (!coords || !split) return fail(COFFEE_ERR_INVALID_ARG, "split_coords: coords and split must be non-NULL");
  if ((reinterpret_cast<uintptr_t>(coords) & 7u) || (reinterpret_cast<uintptr_t>(split) & 7u))
    return fail(COFFEE_ERR_INVALID_ARG, "split_coords: coords and split must be 8-byte aligned");
  DeviceCache* c = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    int rc = device_cache(&c);
    if (rc != COFFEE_OK) return rc;
  }
  const int64_t blocks = std::min<int64_t>((n / 2 + 255) / 256 + 1, (int64_t)c->num_sms * 8);
  k_split_coords<<<(unsigned)blocks, 256, 0, stream>>>(coords, n, reinterpret_cast<float2*>(split));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "launch(split_coords)");
  return COFFEE_OK;
}

int coffee_assemble_ex(const coffee_assemble_args* a, coffee_stream_t stream) {
  return assemble_impl(a, nullptr, 0, stream);
}

int coffee_sparsity(const int32_t* l2g, int64_t ncells, int nloc, int64_t nrows, int64_t* rowptr,
                    int32_t* colidx, int64_t* nnz, coffee_stream_t stream) {
  if (ncells < 0 || nrows < 0 || nloc < 1 || nloc > 128)
    return fail(COFFEE_ERR_INVALID_ARG, "need ncells >= 0, nrows >= 0, 1 <= nloc <= 128");
  if (ncells > INT32_MAX || nrows > INT32_MAX)
    return fail(COFFEE_ERR_INVALID_ARG, "ncells and nrows must fit in int32");
  if (!rowptr || (!colidx && !nnz) || (ncells > 0 && !l2g))
    return fail(COFFEE_ERR_INVALID_ARG, "l2g, rowptr and (colidx or nnz) must be non-NULL");
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceCache* c = nullptr;
  int rc = device_cache(&c);
  if (rc != COFFEE_OK) return rc;
  cudaStream_t s = stream;
  if (ncells == 0 || nrows == 0) {
    if (!colidx) {
      cudaError_t e = cudaMemsetAsync(rowptr, 0, sizeof(int64_t) * (size_t)(nrows + 1), s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(rowptr)");
      *nnz = 0;
    }
    return COFFEE_OK;
  }
  uint8_t* ws = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&ws), sparsity_scratch_bytes(ncells, nloc, nrows), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(sparsity scratch)");
  unsigned* flag = nullptr;
  e = (cudaError_t)launch_sparsity(l2g, ncells, nloc, nrows, rowptr, colidx, ws, &flag, c->num_sms, s);
  unsigned hflag = 0;
  int64_t total = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && !colidx)
    e = cudaMemcpyAsync(&total, rowptr + nrows, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  cudaError_t e2 = cudaFreeAsync(ws, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "sparsity");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync(sparsity scratch)");
  if (hflag & ERR_CAPACITY)
    return fail(COFFEE_ERR_UNSUPPORTED, "a row gathers more than 4096 entries (sum of nloc over its incident cells)");
  if (hflag & ERR_INDEX)
    return fail(COFFEE_ERR_INVALID_ARG, colidx ? "rowptr does not match l2g (count with colidx = NULL first)"
                                               : "an l2g entry is outside [0, nrows)");
  if (!colidx) *nnz = total;
  return COFFEE_OK;
}

int coffee_csr_map(const int32_t* l2g, int64_t ncells, int nloc, const int64_t* rowptr, const int32_t* colidx,
                   int64_t nrows, uint32_t* map, coffee_stream_t stream) {
  if (ncells < 0 || nrows < 0 || nloc < 1 || nloc > 128)
    return fail(COFFEE_ERR_INVALID_ARG, "need ncells >= 0, nrows >= 0, 1 <= nloc <= 128");
  if (ncells == 0) return COFFEE_OK;
  if (!l2g || !rowptr || !colidx || !map) return fail(COFFEE_ERR_INVALID_ARG, "pointers must be non-NULL");
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceCache* c = nullptr;
  int rc = device_cache(&c);
  if (rc != COFFEE_OK) return rc;
  cudaError_t e = (cudaError_t)launch_csr_map(l2g, ncells, nloc, rowptr, colidx, nrows, map, c->err, c->num_sms,
                                              stream);
  if (e != cudaSuccess) return cuda_fail(e, "launch(csr_map)");
  return COFFEE_OK;
}

int coffee_csr_supported(int form, int degree, int cell, int precision) {
  if (!valid_fdc(form, degree, cell) || precision < PREC_FP64 || precision > PREC_BF16X3) return 0;
  if (form == FORM_BURGERS_RES) return 0;
  if (cell == CELL_PRISM)
    return precision == PREC_FP64 ? 1 : prism_tc_supported(form, degree, precision);
  return precision == PREC_FP64 ? 1 : tc_csr_supported(form, degree, cell, precision);
}

int coffee_assemble_csr(const coffee_assemble_args* a, const uint32_t* map, void* vals, int64_t nnz,
                        coffee_stream_t stream) {
  if (!a) return fail(COFFEE_ERR_INVALID_ARG, "args is NULL");
  if (a->ncells > 0 && (!map || !vals)) return fail(COFFEE_ERR_INVALID_ARG, "map and vals must be non-NULL");
  if (nnz < 0 || nnz > (int64_t)UINT32_MAX) return fail(COFFEE_ERR_INVALID_ARG, "nnz must be in [0, 2^32)");
  if (reinterpret_cast<uintptr_t>(map) % 16 != 0) return fail(COFFEE_ERR_INVALID_ARG, "map must be 16-byte aligned");
  if (a->form == FORM_BURGERS_RES)
    return fail(COFFEE_ERR_INVALID_ARG, "the Burgers residual is an element vector, not a matrix");
  coffee_assemble_args b = *a;
  b.out = vals;
  return assemble_impl(&b, map, nnz, stream);
}

int coffee_assemble(int form, int degree, int cell, const double* coords, const int32_t* cell2vert,
                    const double* coef, const int32_t* cell2dof, void* out, int64_t ncells,
                    coffee_stream_t stream) {
  coffee_assemble_args a{};
  a.form = form;
  a.degree = degree;
  a.cell = cell;
  a.precision = COFFEE_FP64;
  a.nu = 0.01;
  a.coords = coords;
  a.nverts = 0;
  a.cell2vert = cell2vert;
  a.coef = coef;
  a.ncoefnodes = INT64_MAX;
  a.cell2dof = cell2dof;
  a.out = out;
  a.ncells = ncells;
  a.flags = 0;
  return coffee_assemble_ex(&a, stream);
}

int coffee_assemble_backward(const coffee_assemble_args* a, const void* dout, double* d_coords,
                             double* d_coef, int deterministic, coffee_stream_t stream) {
  int rc = check_args(a);
  if (rc != COFFEE_OK || a->ncells == 0) return rc;
  if (burgers_like(a->form))
    return fail(COFFEE_ERR_UNSUPPORTED, "no GPU adjoint for the Burgers forms");
  if (a->cell == CELL_PRISM) return fail(COFFEE_ERR_UNSUPPORTED, "no GPU adjoint on prisms");
  if (!dout || !d_coords) return fail(COFFEE_ERR_INVALID_ARG, "dout and d_coords must be non-NULL");
  if (deterministic && (a->nverts <= 0 || (a->form == FORM_ADVDIFF && d_coef && a->ncoefnodes <= 0)))
    return fail(COFFEE_ERR_INVALID_ARG, "deterministic mode needs nverts (and ncoefnodes)");
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceCache* c = nullptr;
  if ((rc = device_cache(&c)) != COFFEE_OK) return rc;
  const double* T = nullptr;
  if ((rc = fp64_table(*c, a->form, a->degree, a->cell, &T)) != COFFEE_OK) return rc;
  const int d = a->cell == CELL_TRI ? 2 : 3;
  const int ns = nnodes(a->cell, a->degree);
  BwdParams p{};
  p.coords = a->coords;
  p.c2v = a->cell2vert;
  p.coef = a->coef;
  p.c2d = a->cell2dof;
  p.T = T;
  p.dout = dout;
  p.dout_fp32 = a->precision != PREC_FP64;
  p.d_coords = d_coords;
  p.d_coef = a->form == FORM_ADVDIFF ? d_coef : nullptr;
  p.err = c->err;
  p.ncells = a->ncells;
  p.nverts = a->nverts;
  p.ncoefnodes = a->ncoefnodes;
  p.N = ns * ns;
  p.validate = (a->flags & COFFEE_FLAG_VALIDATE) ? 1 : 0;
  cudaStream_t s = stream;
  if (!deterministic) {
    cudaError_t e = (cudaError_t)launch_backward(a->form, a->cell, p, s);
    if (e != cudaSuccess) return cuda_fail(e, "launch(assemble_backward)");
    return COFFEE_OK;
  }
  // deterministic: per-cell contributions, then per-node sums in increasing cell order.
  // Scratch is stream-ordered (cudaMallocAsync / cudaFreeAsync on `stream`).
  const int nl = bwd_local_len(a->form, a->cell);
  const int64_t nn = std::max<int64_t>(a->nverts, p.d_coef ? a->ncoefnodes : 0);
  const int64_t width = d + 1;
  const size_t b_local = sizeof(double) * (size_t)a->ncells * nl;
  const size_t b_cnt = sizeof(int32_t) * (size_t)nn;
  const size_t b_off = sizeof(int64_t) * (size_t)(nn + 1);
  const size_t b_slots = sizeof(int64_t) * (size_t)(a->ncells * width);
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t total = al(b_local) + 2 * al(b_cnt) + al(b_off) + al(b_slots);
  uint8_t* ws = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&ws), total, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(backward scratch)");
  double* local = reinterpret_cast<double*>(ws);
  int32_t* cnt = reinterpret_cast<int32_t*>(ws + al(b_local));
  int32_t* cur = reinterpret_cast<int32_t*>(ws + al(b_local) + al(b_cnt));
  int64_t* off = reinterpret_cast<int64_t*>(ws + al(b_local) + 2 * al(b_cnt));
  int64_t* slots = reinterpret_cast<int64_t*>(ws + al(b_local) + 2 * al(b_cnt) + al(b_off));
  p.local = local;
  e = (cudaError_t)launch_backward(a->form, a->cell, p, s);
  if (e == cudaSuccess)
    e = (cudaError_t)launch_ordered_sum(a->cell2vert, a->ncells, (int)width, a->nverts, local, nl, 0, d,
                                        d_coords, d, 0, cnt, cur, off, slots, c->err, s);
  if (e == cudaSuccess && p.d_coef) {
    e = (cudaError_t)launch_ordered_sum(a->cell2dof, a->ncells, (int)width, a->ncoefnodes, local, nl,
                                        (d + 1) * d, 1, d_coef, d + 1, 0, cnt, cur, off, slots, c->err, s);
    if (e == cudaSuccess)
      e = (cudaError_t)launch_ordered_sum(a->cell2dof, a->ncells, (int)width, a->ncoefnodes, local, nl,
                                          (d + 1) * d + (d + 1), d, d_coef, d + 1, 1, cnt, cur, off, slots,
                                          c->err, s);
  }
  cudaError_t e2 = cudaFreeAsync(ws, s);
  if (e != cudaSuccess) return cuda_fail(e, "launch(deterministic backward)");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync(backward scratch)");
  return COFFEE_OK;
}

int coffee_check_errors(coffee_stream_t stream) {
  DeviceCache* c = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    int rc = device_cache(&c);
    if (rc != COFFEE_OK) return rc;
  }
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  unsigned w = 0;
  e = cudaMemcpy(&w, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(error word)");
  if (w) {
    e = cudaMemset(c->err, 0, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(error word)");
  }
  unsigned wn = 0;  // the allocation-free adjoint keeps its own word in its static scratch
  int rc = noalloc_error_word(&wn);
  if (rc != COFFEE_OK) return rc;
  w |= wn;
  if (w & ERR_TIMEOUT) return fail(COFFEE_ERR_TIMEOUT, "a device wait gave up (bounded spin)");
  if (w & ERR_INDEX) return fail(COFFEE_ERR_DEVICE_INDEX, "out-of-range index in cell2vert/cell2dof");
  return COFFEE_OK;
}

const char* coffee_last_error(void) { return g_last_error.c_str(); }

int coffee_table_image(int form, int degree, int cell, int precision, uint8_t* img, int64_t* nbytes,
                       int64_t* meta) {
  if (!nbytes) return fail(COFFEE_ERR_INVALID_ARG, "nbytes is NULL");
  if (precision == PREC_FP64 || !coffee_supported(form, degree, cell, precision))
    return fail(COFFEE_ERR_UNSUPPORTED, "no tensor-core kernel for this form/degree/cell/precision");
  std::vector<uint8_t> h;
  TcTable m{};
  build_tc_image(form, degree, cell, precision, h, m);
  *nbytes = (int64_t)h.size();
  if (meta) {
    const int64_t v[8] = {m.mtiles, m.kbytes, m.kelems, m.K, m.tparts, m.aexact, m.ksteps_off, m.scale_off};
    std::memcpy(meta, v, sizeof v);
  }
  if (img) std::memcpy(img, h.data(), h.size());
  return COFFEE_OK;
}

int coffee_diag_wait_timeout(coffee_stream_t stream) {
  DeviceCache* c = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    int rc = device_cache(&c);
    if (rc != COFFEE_OK) return rc;
  }
  cudaError_t e = (cudaError_t)launch_diag_wait(c->err, stream);
  if (e != cudaSuccess) return cuda_fail(e, "launch(diag_wait)");
  return COFFEE_OK;
}

namespace {
struct BatchPlanImpl {
  BatchLaunch L{};
  BatchGroup* d_groups = nullptr;
  int64_t* d_ranges = nullptr;
  SimtGroup* d_sgroups = nullptr;  // the CUDA-core groups
  int nsg = 0;
  int64_t stiles = 0;
  int num_sms = 0;
  int device = 0;
};
}  // namespace

namespace {
// Contiguous ranges of about equal cost: CTA b takes items [ranges[b], ranges[b+1]), cut after
// the first item at which the running cost reaches b/grid of the total.
void split_by_cost(const double* cost, int64_t items, int grid, int64_t* ranges) {
  double total = 0.0;
  for (int64_t i = 0; i < items; ++i) total += cost[i];
  for (int b = 0; b <= grid; ++b) ranges[b] = items;
  ranges[0] = 0;
  double acc = 0.0;
  int b = 1;
  for (int64_t i = 0; i < items && b < grid; ++i) {
    acc += cost[i];
    if (acc >= total * b / grid) ranges[b++] = i + 1;
  }
}

// Plan shared by both entry points: tile_cost (per group, one full 128-cell tile) when given,
// else bytes written + item_overhead per 128-output slice.
int batch_plan_impl(const coffee_assemble_args* groups, int ngroups, int grid, double item_overhead,
                    const double* tile_cost, void** plan) {
  if (!plan) return fail(COFFEE_ERR_INVALID_ARG, "plan is NULL");
  *plan = nullptr;
  if (!groups || ngroups <= 0) return fail(COFFEE_ERR_INVALID_ARG, "no groups");
  const int prec = groups[0].precision;
  if (prec == PREC_FP64) return fail(COFFEE_ERR_UNSUPPORTED, "batches run on the tensor cores (not FP64)");
  for (int i = 0; i < ngroups; ++i) {
    int rc = check_args(&groups[i]);
    if (rc != COFFEE_OK) return rc;
    if (groups[i].precision != prec) return fail(COFFEE_ERR_INVALID_ARG, "all groups must share one precision");
    if (burgers_like(groups[i].form) || groups[i].cell == CELL_PRISM)
      return fail(COFFEE_ERR_UNSUPPORTED, "the mixed batch covers MASS, HELMHOLTZ and ADVDIFF on simplices");
  }
  if (item_overhead < 0) item_overhead = 16384.0;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceCache* c = nullptr;
  int rc = device_cache(&c);
  if (rc != COFFEE_OK) return rc;
  std::vector<BatchGroup> hg;
  std::vector<SimtGroup> sg;
  std::vector<double> cost;  // per work item
  int kbytes_max = 32;
  int64_t items = 0, stiles = 0;
  const bool all_tc = (groups[0].flags & COFFEE_FLAG_TENSOR_CORES) != 0;
  for (int i = 0; i < ngroups; ++i) {
    const coffee_assemble_args* a = &groups[i];
    const int ns = nnodes(a->cell, a->degree);
    if (!all_tc && simt_supported(a->form, a->degree, a->cell) && simt_default(a->form, a->degree, a->cell)) {
      // CUDA-core group: the standalone kernel's parameters, warp tiles numbered on
      cudaError_t eu = (cudaError_t)simt_upload(a->form, a->degree, a->cell);
      if (eu != cudaSuccess) return cuda_fail(eu, "coffee_batch_plan (reference tensor)");
      SimtGroup s{};
      s.p.coords = a->coords;
      s.p.c2v = a->cell2vert;
      s.p.coef = a->coef;
      s.p.c2d = a->cell2dof;
      s.p.out = static_cast<float*>(a->out);
      s.p.err = c->err;
      s.p.ncells = a->ncells;
      s.p.nverts = a->nverts;
      s.p.ncoefnodes = a->ncoefnodes;
      s.p.ns = ns;
      s.p.N = ns * ns;
      s.p.ostride = ns * ns;
      s.p.precision = prec;
      s.p.xs = a->coords_split;
      s.p.cf = a->coef_f32;
      s.p.validate = (a->flags & COFFEE_FLAG_VALIDATE) ? 1 : 0;
      s.p.nu = a->nu;
      s.tile0 = stiles;
      s.kind = simt_kind(a->form, a->degree, a->cell);
      stiles += (a->ncells + 31) / 32;
      sg.push_back(s);
      continue;
    }
    TcTable meta{};
    if ((rc = tc_table(*c, a->form, a->degree, a->cell, prec, &meta)) != COFFEE_OK) return rc;
    hg.emplace_back();
    BatchGroup& g = hg.back();
    std::memset(&g, 0, sizeof(g));
    g.p.coords = a->coords;
    g.p.c2v = a->cell2vert;
    g.p.coef = a->coef;
    g.p.c2d = a->cell2dof;
    g.p.image = meta.image;
    g.p.out = static_cast<float*>(a->out);
    g.p.err = c->err;
    g.p.ncells = a->ncells;
    g.p.nverts = a->nverts;
    g.p.ncoefnodes = a->ncoefnodes;
    g.p.ns = ns;
    g.p.N = ns * ns;
    g.p.ostride = ns * ns;  // batches write contiguous rows
    g.p.mtiles = meta.mtiles;
    g.p.kbytes = meta.kbytes;
    g.p.tparts = meta.tparts;
    g.p.precision = prec;
    g.p.xs = a->coords_split;
    g.p.cf = a->coef_f32;
    g.p.validate = (a->flags & COFFEE_FLAG_VALIDATE) ? 1 : 0;
    g.p.nu = a->nu;
    g.item0 = items;
    g.form = a->form;
    g.cell = a->cell;
    g.degree = a->degree;
    g.lanes = g.p.N <= 32 ? 1 : 0;
    kbytes_max = std::max(kbytes_max, meta.kbytes);
    const int64_t nt = (a->ncells + 127) / 128;
    for (int64_t t = 0; t < nt; ++t) {
      const int64_t cells = std::min<int64_t>(128, a->ncells - t * 128);
      cost.push_back(tile_cost ? tile_cost[i] * (double)cells / 128.0
                               : 4.0 * (double)cells * g.p.N + item_overhead * meta.mtiles);
    }
    items += nt;
  }
  if (items == 0 && stiles == 0) return fail(COFFEE_ERR_INVALID_ARG, "all groups are empty");
  const int ntc = (int)hg.size();
  int nstages = 0, smem = 0;
  if (items > 0) {
    smem = batch_smem(kbytes_max, prec, &nstages);
    if (smem == 0) return fail(COFFEE_ERR_UNSUPPORTED, "batch operands do not fit in shared memory");
  }
  if (grid <= 0) grid = c->num_sms;
  grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, items));
  std::vector<int64_t> ranges(grid + 1, 0);
  if (items > 0) split_by_cost(cost.data(), items, grid, ranges.data());
  auto* P = new BatchPlanImpl();
  cudaGetDevice(&P->device);
  cudaError_t e = cudaSuccess;
  if (ntc > 0) {
    e = cudaMalloc(&P->d_groups, sizeof(BatchGroup) * ntc);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_ranges, sizeof(int64_t) * (grid + 1));
    if (e == cudaSuccess) e = cudaMemcpy(P->d_groups, hg.data(), sizeof(BatchGroup) * ntc, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(P->d_ranges, ranges.data(), sizeof(int64_t) * (grid + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = (cudaError_t)batch_prepare(prec, smem);
  }
  if (e == cudaSuccess && !sg.empty()) {
    e = cudaMalloc(&P->d_sgroups, sizeof(SimtGroup) * sg.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(P->d_sgroups, sg.data(), sizeof(SimtGroup) * sg.size(), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cudaFree(P->d_groups);
    cudaFree(P->d_ranges);
    cudaFree(P->d_sgroups);
    delete P;
    return cuda_fail(e, "coffee_batch_plan");
  }
  P->nsg = (int)sg.size();
  P->stiles = stiles;
  P->num_sms = c->num_sms;
  P->L.groups = P->d_groups;
  P->L.ngroups = ntc;
  P->L.ranges = P->d_ranges;
  P->L.grid = grid;
  P->L.smem = smem;
  P->L.nstages = nstages;
  P->L.kbytes_max = kbytes_max;
  P->L.precision = prec;
  P->L.err = c->err;
  *plan = P;
  return COFFEE_OK;
}
}  // namespace

int coffee_batch_plan(const coffee_assemble_args* groups, int ngroups, int grid, double item_overhead,
                      void** plan) {
  return batch_plan_impl(groups, ngroups, grid, item_overhead, nullptr, plan);
}

int coffee_batch_plan_costs(const coffee_assemble_args* groups, int ngroups, int grid, const double* tile_cost,
                            void** plan) {
  if (!tile_cost) return fail(COFFEE_ERR_INVALID_ARG, "tile_cost is NULL");
  for (int i = 0; i < ngroups; ++i)
    if (!(tile_cost[i] > 0.0) || !std::isfinite(tile_cost[i]))
      return fail(COFFEE_ERR_INVALID_ARG, "tile_cost must be positive and finite");
  return batch_plan_impl(groups, ngroups, grid, -1.0, tile_cost, plan);
}

int coffee_batch_split(const double* cost, int64_t items, int grid, int64_t* ranges) {
  if (items < 0 || grid < 1) return fail(COFFEE_ERR_INVALID_ARG, "need items >= 0 and grid >= 1");
  if (!ranges || (items > 0 && !cost)) return fail(COFFEE_ERR_INVALID_ARG, "cost and ranges must be non-NULL");
  for (int64_t i = 0; i < items; ++i)
    if (!(cost[i] >= 0.0) || !std::isfinite(cost[i]))
      return fail(COFFEE_ERR_INVALID_ARG, "costs must be finite and >= 0");
  split_by_cost(cost, items, grid, ranges);
  return COFFEE_OK;
}

int coffee_batch_launch(void* plan, coffee_stream_t stream) {
  if (!plan) return fail(COFFEE_ERR_INVALID_ARG, "plan is NULL");
  auto* P = static_cast<BatchPlanImpl*>(plan);
  if (P->nsg > 0) {
    cudaError_t e = (cudaError_t)launch_simt_batch(P->d_sgroups, P->nsg, P->stiles, P->num_sms, stream);
    if (e != cudaSuccess) return cuda_fail(e, "launch(batch, CUDA cores)");
  }
  if (P->L.ngroups > 0) {
    cudaError_t e = (cudaError_t)batch_launch(P->L, stream);
    if (e != cudaSuccess) return cuda_fail(e, "launch(batch)");
  }
  return COFFEE_OK;
}

void coffee_batch_free(void* plan) {
  if (!plan) return;
  auto* P = static_cast<BatchPlanImpl*>(plan);
  cudaFree(P->d_groups);
  cudaFree(P->d_ranges);
  cudaFree(P->d_sgroups);
  delete P;
}

}  // extern "C"
