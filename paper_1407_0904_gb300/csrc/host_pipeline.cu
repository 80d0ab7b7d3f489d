// Local assembly of host-resident data (coffee_assemble_host): the copies around
// coffee_assemble_ex. Coordinates and coefficients go to the device once (for the tensor-core
// precisions on simplices the coordinates are then split into (hi, lo) float pairs on the
// device, coffee_split_coords); the cells are
// assembled in chunks, each chunk's index rows copied in on the caller's stream before its
// launch and its element matrices copied back on a library-owned stream while the next
// chunk computes. Staging memory comes from a library-owned stream-ordered pool.
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include "../../include/coffee.h"
#include "coffee_internal.h"

namespace coffee {
namespace {

struct HostRes {
  cudaStream_t side = nullptr;   // device-to-host copies
  cudaMemPool_t pool = nullptr;  // staging buffers, kept for reuse
};

std::mutex h_mu;
std::map<int, HostRes> h_res;

int cuda_err(cudaError_t e, const char* where) {
  return fail(COFFEE_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int host_res(HostRes** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lock(h_mu);
  HostRes& r = h_res[dev];
  if (!r.side) {
    e = cudaStreamCreateWithFlags(&r.side, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      r.side = nullptr;
      return cuda_err(e, "cudaStreamCreateWithFlags");
    }
  }
  if (!r.pool) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    e = cudaMemPoolCreate(&r.pool, &props);
    if (e != cudaSuccess) {
      r.pool = nullptr;
      return cuda_err(e, "cudaMemPoolCreate");
    }
    uint64_t keep = UINT64_MAX;  // no release at synchronisation points: the next call reuses it
    e = cudaMemPoolSetAttribute(r.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) return cuda_err(e, "cudaMemPoolSetAttribute");
  }
  *out = &r;
  return COFFEE_OK;
}

}  // namespace
}  // namespace coffee

using namespace coffee;

extern "C" {

int coffee_assemble_host(const coffee_assemble_args* a, int chunks, coffee_stream_t stream) {
  if (!a) return fail(COFFEE_ERR_INVALID_ARG, "args is NULL");
  if (chunks < 1) return fail(COFFEE_ERR_INVALID_ARG, "chunks must be >= 1");
  if (a->ncells < 0) return fail(COFFEE_ERR_INVALID_ARG, "ncells < 0");
  if (!coffee_supported(a->form, a->degree, a->cell, a->precision))
    return fail(COFFEE_ERR_UNSUPPORTED, "no kernel for this form/degree/cell/precision");
  if (a->ncells == 0) return COFFEE_OK;
  if (!a->coords || !a->cell2vert || !a->out)
    return fail(COFFEE_ERR_INVALID_ARG, "coords, cell2vert and out must be non-NULL");
  if (a->nverts <= 0) return fail(COFFEE_ERR_INVALID_ARG, "nverts must be > 0 (it sizes the coordinate copy)");
  if (a->out_stride != 0) return fail(COFFEE_ERR_INVALID_ARG, "out_stride must be 0 for host buffers");
  const bool has_coef = a->form == FORM_ADVDIFF || burgers_like(a->form);
  if (has_coef && (!a->coef || !a->cell2dof || a->ncoefnodes <= 0))
    return fail(COFFEE_ERR_INVALID_ARG, "this form needs coef, cell2dof and ncoefnodes > 0");
  const int n = coffee_ndof(a->form, a->degree, a->cell);
  if (n < 0) return n;

  // byte sizes of every array (layouts of coffee_assemble)
  const int d = a->cell == CELL_TRI ? 2 : 3;
  const int nv = a->cell == CELL_TRI ? 3 : a->cell == CELL_TET ? 4 : 6;
  const int w = a->form == FORM_ADVDIFF ? nv : burgers_like(a->form) ? nnodes(a->cell, a->degree) : 0;
  const size_t coef_row = a->form == FORM_ADVDIFF ? (size_t)(1 + d) : (size_t)d;
  const size_t row_out = (size_t)(a->form == FORM_BURGERS_RES ? n : n * n) * (a->precision == PREC_FP64 ? 8 : 4);
  const int64_t nc = a->ncells;
  const size_t b_coords = (size_t)a->nverts * d * sizeof(double);
  const size_t b_coef = has_coef ? (size_t)a->ncoefnodes * coef_row * sizeof(double) : 0;
  const size_t b_c2v = (size_t)nc * nv * sizeof(int32_t), b_c2d = (size_t)nc * w * sizeof(int32_t);
  const size_t b_out = (size_t)nc * row_out;
  // tensor-core kernels on simplices take the vertex differences from (hi, lo) float pairs
  const bool split = a->precision != PREC_FP64 && a->cell != CELL_PRISM;
  const size_t b_split = split ? (size_t)a->nverts * d * 2 * sizeof(float) : 0;
  // and every tensor-core kernel takes the coefficients as floats, rounded once per node
  const bool round = a->precision != PREC_FP64 && has_coef;
  const size_t b_cf = round ? (size_t)a->ncoefnodes * coef_row * sizeof(float) : 0;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_coef = al(b_coords), o_c2v = o_coef + al(b_coef), o_c2d = o_c2v + al(b_c2v),
               o_out = o_c2d + al(b_c2d), o_split = o_out + al(b_out), o_cf = o_split + al(b_split),
               total = o_cf + al(b_cf);

  HostRes* r = nullptr;
  int rc = host_res(&r);
  if (rc != COFFEE_OK) return rc;
  cudaStream_t s = stream;
  uint8_t* ws = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&ws), total, r->pool, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(COFFEE_ERR_NOMEM, std::string("staging buffers (") + std::to_string(total) +
                                      " bytes): " + cudaGetErrorString(e));
  }
  double* d_coords = reinterpret_cast<double*>(ws);
  double* d_coef = has_coef ? reinterpret_cast<double*>(ws + o_coef) : nullptr;
  int32_t* d_c2v = reinterpret_cast<int32_t*>(ws + o_c2v);
  int32_t* d_c2d = has_coef ? reinterpret_cast<int32_t*>(ws + o_c2d) : nullptr;
  uint8_t* d_out = ws + o_out;
  float* d_split = split ? reinterpret_cast<float*>(ws + o_split) : nullptr;
  float* d_cf = round ? reinterpret_cast<float*>(ws + o_cf) : nullptr;
  uint8_t* h_out = static_cast<uint8_t*>(a->out);

  e = cudaMemcpyAsync(d_coords, a->coords, b_coords, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && has_coef) e = cudaMemcpyAsync(d_coef, a->coef, b_coef, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) rc = cuda_err(e, "cudaMemcpyAsync(coordinates, coefficients)");
  if (rc == COFFEE_OK && split) rc = coffee_split_coords(d_coords, a->nverts * d, d_split, s);
  if (rc == COFFEE_OK && round) rc = coffee_round_coef(d_coef, a->ncoefnodes * (int64_t)coef_row, d_cf, s);

  // chunks of whole 128-cell tiles, so every chunk's output starts 512-byte aligned
  int64_t per = (nc + chunks - 1) / chunks;
  per = (per + 127) / 128 * 128;
  for (int64_t lo = 0; lo < nc && rc == COFFEE_OK; lo += per) {
    const int64_t hi = std::min(nc, lo + per), m = hi - lo;
    e = cudaMemcpyAsync(d_c2v + lo * nv, a->cell2vert + lo * nv, (size_t)m * nv * sizeof(int32_t),
                        cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && has_coef)
      e = cudaMemcpyAsync(d_c2d + lo * w, a->cell2dof + lo * w, (size_t)m * w * sizeof(int32_t),
                          cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      rc = cuda_err(e, "cudaMemcpyAsync(index rows)");
      break;
    }
    coffee_assemble_args b = *a;
    b.coords = d_coords;
    b.coords_split = d_split;
    b.coef = d_coef;
    b.coef_f32 = d_cf;
    b.cell2vert = d_c2v + lo * nv;
    b.cell2dof = has_coef ? d_c2d + lo * w : nullptr;
    b.out = d_out + (size_t)lo * row_out;
    b.ncells = m;
    rc = coffee_assemble_ex(&b, s);
    if (rc != COFFEE_OK) break;
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(r->side, ev, 0);
    if (ev) cudaEventDestroy(ev);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_out + (size_t)lo * row_out, d_out + (size_t)lo * row_out, (size_t)m * row_out,
                          cudaMemcpyDeviceToHost, r->side);
    if (e != cudaSuccess) rc = cuda_err(e, "chunk hand-off or cudaMemcpyAsync(results)");
  }

  // the caller's stream waits for the last copy back, then the staging memory returns to the pool
  cudaEvent_t done = nullptr;
  e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(done, r->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, done, 0);
  if (done) cudaEventDestroy(done);
  if (e != cudaSuccess) {
    // without the join the staging memory cannot be released in stream order: wait instead
    cudaStreamSynchronize(r->side);
    if (rc == COFFEE_OK) rc = cuda_err(e, "joining the copy stream");
  }
  cudaError_t ef = cudaFreeAsync(ws, s);
  if (ef != cudaSuccess && rc == COFFEE_OK) rc = cuda_err(ef, "cudaFreeAsync(staging buffers)");
  return rc;
}

int coffee_host_pool_trim(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return COFFEE_OK;
  std::lock_guard<std::mutex> lock(h_mu);
  auto it = h_res.find(dev);
  if (it != h_res.end() && it->second.pool) cudaMemPoolTrimTo(it->second.pool, 0);
  return COFFEE_OK;
}

}  // extern "C"
