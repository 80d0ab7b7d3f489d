// Allocation-free variant of the deterministic adjoint (coffee_assemble_backward_noalloc).
//
// Who needs it: callers that must not allocate device memory while they run. cudaMalloc
// and cudaFree can synchronise the whole device and stall other streams, so latency-
// critical loops avoid them; some applications hand all device memory to their own
// pool or caching allocator and forbid allocation by libraries; embedded and
// fixed-budget deployments must know every device byte up front. The regular
// deterministic adjoint takes stream-ordered scratch from cudaMallocAsync and its
// reference tensors from a lazily allocated cache; this entry point instead keeps all
// of its scratch in one file-scope device array of fixed size, reserved on every GPU
// that loads the library until the process exits.
//
// Scratch layout (each region 256-byte aligned), sized for at most
// NOALLOC_MAX_CELLS cells and NOALLOC_MAX_NODES vertices / coefficient nodes:
//   per-cell contributions [cells][28] double | FP64 reference tensor [36*1225] double |
//   node counts, cursors [nodes] int32 | segment offsets [nodes+1] int64 |
//   segment slots [cells*4] int64 | error word (read and cleared by coffee_check_errors).
#include <cuda_runtime.h>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>
#include "../../include/coffee.h"
#include "coffee_internal.h"

namespace coffee {
namespace {

constexpr int64_t NOALLOC_MAX_CELLS = 16384;
constexpr int64_t NOALLOC_MAX_NODES = 16384;
constexpr int NL_MAX = 28;              // longest per-cell gradient: advection-diffusion on tets
constexpr int64_t T_MAX = 36 * 1225;    // largest FP64 reference tensor: advection-diffusion, tet P4

constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t R_LOCAL = al256(sizeof(double) * NOALLOC_MAX_CELLS * NL_MAX);
constexpr size_t R_T = al256(sizeof(double) * T_MAX);
constexpr size_t R_CNT = al256(sizeof(int32_t) * NOALLOC_MAX_NODES);
constexpr size_t R_OFF = al256(sizeof(int64_t) * (NOALLOC_MAX_NODES + 1));
constexpr size_t R_SLOTS = al256(sizeof(int64_t) * NOALLOC_MAX_CELLS * 4);
constexpr size_t R_ERR = 256;
constexpr size_t O_LOCAL = 0;
constexpr size_t O_T = O_LOCAL + R_LOCAL;
constexpr size_t O_CNT = O_T + R_T;
constexpr size_t O_CUR = O_CNT + R_CNT;
constexpr size_t O_OFF = O_CUR + R_CNT;
constexpr size_t O_SLOTS = O_OFF + R_OFF;
constexpr size_t O_ERR = O_SLOTS + R_SLOTS;
constexpr size_t SCRATCH_BYTES = O_ERR + R_ERR;  // about 4.4 MB

// The scratch itself. In host code this name is only a stand-in for the symbol: its
// device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

std::mutex g_na_mu;
std::map<int, unsigned char*> g_na_addr;                               // device -> scratch address
std::map<std::tuple<int, int, int>, std::vector<double>> g_na_tables;  // host copies of T
std::map<int, std::tuple<int, int, int>> g_na_resident;                // device -> T held in its scratch

int scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(COFFEE_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  auto it = g_na_addr.find(dev);
  if (it == g_na_addr.end()) {
    unsigned char* ptr = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&ptr), g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr)
      return fail(COFFEE_ERR_CUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e));
    it = g_na_addr.emplace(dev, ptr).first;
  }
  *out = it->second;
  return COFFEE_OK;
}

}  // namespace

// The error word of the no-alloc scratch on the current device (0 when the entry point never
// ran there), read after the caller's synchronisation and cleared when set.
int noalloc_error_word(unsigned* w) {
  *w = 0;
  std::lock_guard<std::mutex> lock(g_na_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return COFFEE_OK;
  auto it = g_na_addr.find(dev);
  if (it == g_na_addr.end()) return COFFEE_OK;
  unsigned* err = reinterpret_cast<unsigned*>(it->second + O_ERR);
  cudaError_t e = cudaMemcpy(w, err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && *w) e = cudaMemset(err, 0, sizeof(unsigned));
  if (e != cudaSuccess) return fail(COFFEE_ERR_CUDA, std::string("no-alloc error word: ") + cudaGetErrorString(e));
  return COFFEE_OK;
}

}  // namespace coffee

using namespace coffee;

extern "C" int coffee_assemble_backward_noalloc(const coffee_assemble_args* a, const void* dout,
                                                double* d_coords, double* d_coef,
                                                coffee_stream_t stream) {
  if (!a) return fail(COFFEE_ERR_INVALID_ARG, "args is NULL");
  if (!(a->form == FORM_MASS || a->form == FORM_HELMHOLTZ || a->form == FORM_ADVDIFF))
    return fail(burgers_like(a->form) ? COFFEE_ERR_UNSUPPORTED : COFFEE_ERR_INVALID_ARG,
                "no-alloc adjoint: form must be MASS, HELMHOLTZ or ADVDIFF");
  if (a->degree < 1 || a->degree > 4 || !(a->cell == CELL_TRI || a->cell == CELL_TET))
    return fail(COFFEE_ERR_INVALID_ARG, "no-alloc adjoint: degree 1..4, triangle or tetrahedron");
  if (a->precision < PREC_FP64 || a->precision > PREC_BF16X3)
    return fail(COFFEE_ERR_INVALID_ARG, "no-alloc adjoint: precision out of range");
  if (a->ncells < 0) return fail(COFFEE_ERR_INVALID_ARG, "no-alloc adjoint: ncells < 0");
  if (a->ncells == 0) return COFFEE_OK;
  if (a->flags & COFFEE_FLAG_VALIDATE)
    return fail(COFFEE_ERR_INVALID_ARG,
                "no-alloc adjoint: COFFEE_FLAG_VALIDATE is not supported (validate with coffee_assemble_backward)");
  if (!a->coords || !a->cell2vert || !dout || !d_coords)
    return fail(COFFEE_ERR_INVALID_ARG, "no-alloc adjoint: coords, cell2vert, dout and d_coords must be non-NULL");
  const bool with_coef = a->form == FORM_ADVDIFF && d_coef != nullptr;
  if (a->form == FORM_ADVDIFF && (!a->coef || !a->cell2dof))
    return fail(COFFEE_ERR_INVALID_ARG, "no-alloc adjoint: ADVDIFF needs coef and cell2dof");
  if (a->ncells > NOALLOC_MAX_CELLS)
    return fail(COFFEE_ERR_INVALID_ARG, "no-alloc adjoint: ncells exceeds the fixed scratch limit of 16384 cells");
  if (a->nverts <= 0 || a->nverts > NOALLOC_MAX_NODES)
    return fail(COFFEE_ERR_INVALID_ARG, "no-alloc adjoint: nverts must be in 1..16384 (fixed scratch limit)");
  if (with_coef && (a->ncoefnodes <= 0 || a->ncoefnodes > NOALLOC_MAX_NODES))
    return fail(COFFEE_ERR_INVALID_ARG, "no-alloc adjoint: ncoefnodes must be in 1..16384 (fixed scratch limit)");

  std::lock_guard<std::mutex> lock(g_na_mu);
  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != COFFEE_OK) return rc;

  // reference tensors: host copy cached per (form, degree, cell), copied into the scratch
  auto key = std::make_tuple(a->form, a->degree, a->cell);
  auto it = g_na_tables.find(key);
  if (it == g_na_tables.end()) {
    std::vector<double> T;
    reference_tensor(a->form, a->degree, a->cell, T);
    it = g_na_tables.emplace(key, std::move(T)).first;
  }
  const std::vector<double>& T = it->second;
  if ((int64_t)T.size() > T_MAX)
    return fail(COFFEE_ERR_UNSUPPORTED, "no-alloc adjoint: reference tensor larger than its scratch region");
  cudaStream_t s = stream;
  double* dT = reinterpret_cast<double*>(base + O_T);
  // the error word starts at zero (static device memory) and keeps its bits until
  // coffee_check_errors reads and clears it, like the library's own error word
  unsigned* err = reinterpret_cast<unsigned*>(base + O_ERR);
  // T is uploaded only when another (form, degree, cell) was last held in this device's
  // scratch: calls are serialised by the caller, so a table left by the previous call is in place
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) {
    auto res = g_na_resident.find(dev);
    if (res == g_na_resident.end() || res->second != key) {
      g_na_resident.erase(dev);
      e = cudaMemcpyAsync(dT, T.data(), T.size() * sizeof(double), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) g_na_resident[dev] = key;
    }
  }
  if (e != cudaSuccess) return fail(COFFEE_ERR_CUDA, std::string("no-alloc adjoint: ") + cudaGetErrorString(e));

  const int d = a->cell == CELL_TRI ? 2 : 3;
  const int ns = nnodes(a->cell, a->degree);
  BwdParams p{};
  p.coords = a->coords;
  p.c2v = a->cell2vert;
  p.coef = a->coef;
  p.c2d = a->cell2dof;
  p.T = dT;
  p.dout = dout;
  p.dout_fp32 = a->precision != PREC_FP64;
  p.d_coords = d_coords;
  p.d_coef = with_coef ? d_coef : nullptr;
  p.local = reinterpret_cast<double*>(base + O_LOCAL);  // every row [0, ncells) is rewritten
  p.err = err;
  p.ncells = a->ncells;
  p.nverts = a->nverts;
  p.ncoefnodes = a->ncoefnodes;
  p.N = ns * ns;
  p.validate = 0;
  const int nl = bwd_local_len(a->form, a->cell);
  int32_t* cnt = reinterpret_cast<int32_t*>(base + O_CNT);  // cleared by launch_ordered_sum
  int32_t* cur = reinterpret_cast<int32_t*>(base + O_CUR);  // cleared by launch_ordered_sum
  int64_t* off = reinterpret_cast<int64_t*>(base + O_OFF);
  int64_t* slots = reinterpret_cast<int64_t*>(base + O_SLOTS);
  e = (cudaError_t)launch_backward(a->form, a->cell, p, s);
  if (e == cudaSuccess)
    e = (cudaError_t)launch_ordered_sum(a->cell2vert, a->ncells, d + 1, a->nverts, p.local, nl, 0, d, d_coords, d,
                                        0, cnt, cur, off, slots, err, s);
  if (e == cudaSuccess && with_coef) {
    e = (cudaError_t)launch_ordered_sum(a->cell2dof, a->ncells, d + 1, a->ncoefnodes, p.local, nl, (d + 1) * d, 1,
                                        d_coef, d + 1, 0, cnt, cur, off, slots, err, s);
    if (e == cudaSuccess)
      e = (cudaError_t)launch_ordered_sum(a->cell2dof, a->ncells, d + 1, a->ncoefnodes, p.local, nl,
                                          (d + 1) * d + (d + 1), d, d_coef, d + 1, 1, cnt, cur, off, slots, err, s);
  }
  if (e != cudaSuccess) return fail(COFFEE_ERR_CUDA, std::string("no-alloc adjoint launch: ") + cudaGetErrorString(e));
  return COFFEE_OK;
}
