/*
 * coffee.h — C ABI of the GB300 finite-element local-assembly library (libcoffee.so).
 *
 * The operation is local assembly as structured in Luporini et al., "COFFEE: an
 * Optimizing Compiler for Finite Element Local Assembly" (arXiv:1407.0904),
 * section 2 ("Structure of a local assembly kernel"; Listings 1 and 2): for every
 * mesh cell, (1) the affine Jacobian J, its determinant and inverse K are computed
 * from the cell's vertex coordinates, (2) basis functions are tabulated at
 * quadrature points on the reference cell, and (3) the element matrix is
 * evaluated by a quadrature loop nest A[j][k] += integrand * det * W[i].
 * Section 3.3 (the outer-product equation) observes that the j-k nest is a sum of
 * outer products; this library pre-sums the quadrature loop into fixed reference
 * tensors T[k][i*n+j] and evaluates A_e = sum_k G_e[k] T[k] as a batched dense
 * contraction over cells (section 5.9 reduces Helmholtz to a few matrix products in
 * the same spirit, one cell at a time).
 *
 * Conventions (the paper leaves them open):
 *  - reference cells: triangle (0,0),(1,0),(0,1); tetrahedron (0,0,0),(1,0,0),
 *    (0,1,0),(0,0,1);
 *  - geometry (pinned by Listing 1): J[r][c] = x_{c+1}[r] - x_0[r], x = x_0 + J xi,
 *    K = J^{-1}, dphi/dx_c = sum_a K[a][c] dphi/dxi_a; the measure is |det J|;
 *  - degree-k Lagrange nodes: lattice points (a,b,c)/k with a+b+c <= k, ordered with
 *    c slowest, then b, then a fastest (degree 1: the vertex order);
 *  - element matrices are [ncells][ndof][ndof] row-major; row = test function,
 *    column = trial function;
 *  - vector-valued (Burgers) dofs are blocked by component: I = c*ns + i.
 *
 * Forms (section 5.2 names Helmholtz, advection-diffusion and Burgers):
 *  MASS        A[i][j] = int phi_i phi_j
 *  HELMHOLTZ   A[i][j] = int grad phi_i . grad phi_j + phi_i phi_j          (Listing 1)
 *  ADVDIFF     A[i][j] = int eps grad phi_i . grad phi_j + phi_i (b . grad phi_j),
 *              eps (scalar) and b (vector) are P1 fields given per coefficient node
 *  BURGERS_JAC A[(ci,i),(cj,j)] = int phi_i phi_j d_cj u_ci
 *                               + [ci==cj] (phi_i (u . grad phi_j) + nu grad phi_i . grad phi_j),
 *              the Jacobian of int (u.grad u).v + nu grad u : grad v for the vector
 *              degree-k field u (Listing 2 is its degree-1 instance)
 *  BURGERS_RESIDUAL  R[(c,i)] = int (u . grad u_c) phi_i + nu grad u_c . grad phi_i, the element
 *              VECTOR of that residual (section 2: local assembly produces element matrices and
 *              element vectors); out is [ncells][d*ns], component-blocked like the Jacobian's rows;
 *              coef and cell2dof as for BURGERS_JAC
 *
 * Ownership: the caller owns every buffer it passes. The library owns only its
 * device cache of reference tensors (created on first use per device, guarded by a
 * mutex, kept until process exit) and batch plans (freed by coffee_batch_free).
 *
 * Errors: every entry point returns a coffee_status. Argument errors are detected
 * on the host before any launch; the message of the last error on the calling
 * thread is returned by coffee_last_error(). Launches are asynchronous on the given
 * stream (NULL = legacy default stream); errors raised while a kernel runs are
 * reported by coffee_check_errors(). No entry point traps on the device.
 */
#ifndef COFFEE_H
#define COFFEE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t (struct CUstream_st*), declared without CUDA headers. */
typedef struct CUstream_st* coffee_stream_t;

/* Prisms (the paper's third element shape): reference triangle x [0,1]; cell2vert rows are
 * the bottom triangle's vertices, then the three vertices above them; degree-k tensor-product
 * Lagrange space (node (a,b,c) at (a/k, b/k, c/k), zeta level c slowest); the map uses the
 * degree-1 prism functions, so it is not affine and the element matrix is the quadrature sum
 * of a fixed rule: n = k+2 Gauss-Legendre points per direction on [0,1], the triangle factor
 * collapsed by (s,t) -> (s, t(1-s)) with weight w_s w_t (1-s). Prisms support MASS, HELMHOLTZ
 * and ADVDIFF (eps and b given per vertex through cell2dof [ncells][6], evaluated at each point
 * with the degree-1 prism functions): FP64 and the tensor-core precisions for P1-P4
 * (the contraction over all quadrature points is streamed through shared memory in K-chunks,
 * at most three 128-output slices at a time),
 * both through coffee_assemble_ex and coffee_assemble_csr. The Burgers Jacobian and residual on
 * prisms (u per node through cell2dof [ncells][(k+1)^2(k+2)/2], rows and columns blocked by
 * component as on simplices) run in FP64 with their own rule of (3k+3)/2 points per direction
 * (the trilinear term's degree), the Jacobian also through coffee_assemble_csr; other
 * precisions return COFFEE_ERR_UNSUPPORTED. */
typedef enum { COFFEE_TRIANGLE = 0, COFFEE_TETRAHEDRON = 1, COFFEE_PRISM = 2 } coffee_cell;

typedef enum {
  COFFEE_MASS = 0,
  COFFEE_HELMHOLTZ = 1,
  COFFEE_ADVDIFF = 2,
  COFFEE_BURGERS_JAC = 3,
  COFFEE_BURGERS_RESIDUAL = 4 /* element vectors, see below */
} coffee_form;

/* Arithmetic of the contraction A_e = sum_k G_e[k] T[k] (per-cell factors G, reference
 * tensors T), accumulated in FP32 on the tensor cores, float output; FP64: CUDA-core FP64,
 * double output. Each operand is held as a sum of parts of the operand type, each part the
 * round-to-nearest of what the previous ones left:
 *   TF32:   T and G one tf32 part each, one product;
 *   TF32X3: T and G two tf32 parts each, the three products hi*hi + hi*lo + lo*hi;
 *   BF16:   T two bf16 parts, G one, two products;
 *   BF16X3: T and G three bf16 parts each, the six products of order <= 2.
 * Parity bounds (max |A - A_exact| / max |A_exact| per cell): 1e-5 for TF32X3 and BF16X3,
 * 1e-2 for TF32 and BF16. */
typedef enum {
  COFFEE_FP64 = 0,
  COFFEE_TF32 = 1,
  COFFEE_TF32X3 = 2,
  COFFEE_BF16 = 3,
  COFFEE_BF16X3 = 4
} coffee_precision;

typedef enum {
  COFFEE_OK = 0,
  COFFEE_ERR_INVALID_ARG = -1,
  COFFEE_ERR_UNSUPPORTED = -2,
  COFFEE_ERR_CUDA = -3,
  COFFEE_ERR_DEVICE_INDEX = -4,
  COFFEE_ERR_NOMEM = -5,
  COFFEE_ERR_TIMEOUT = -6
} coffee_status;

/* Flags of coffee_assemble_args.flags */
#define COFFEE_FLAG_VALIDATE 1u /* range-check cell2vert/cell2dof on the device */
/* Tuning knobs of the tensor-core kernels (results are identical; only speed changes):
 * OUTPUT_LANES: keep element-matrix entries on the TMEM lanes (one 128-output slice per
 *   accumulator) even when the matrix is small enough to put cells on the lanes;
 * TWO_STAGES: at most two operand stages (leaves shared memory to other kernels). */
#define COFFEE_FLAG_OUTPUT_LANES 2u
#define COFFEE_FLAG_TWO_STAGES 4u
/* cells per TMEM accumulator when the outputs are on the lanes (tile shape of the MMA:
 * M = 128 outputs x N = 128, 64 or 32 cells); default 128, or 64 above 512 outputs */
#define COFFEE_FLAG_SUBTILE_64 8u
#define COFFEE_FLAG_SUBTILE_32 16u
#define COFFEE_FLAG_SUBTILE_128 32u
/* cells on the TMEM lanes (M = 128 cells, N = entries) for element matrices of up to 128
 * entries; by default only up to 32 entries */
#define COFFEE_FLAG_CELL_LANES 64u
/* with the outputs on the TMEM lanes, gather whole rows of 8 or 32 consecutive cells in shared
 * memory and write each group with one bulk copy, instead of warp stores of 32 entries of one
 * cell (the default) */
#define COFFEE_FLAG_STAGED_STORE 256u
/* Small element matrices (MASS, HELMHOLTZ, ADVDIFF on triangles P1-P3 and tetrahedra P1-P2;
 * the Burgers Jacobian and residual on P1 simplices and P2 triangles) have a second kernel
 * besides the tensor-core one: one CUDA-core thread per cell, A_e = sum_k G_e[k] T[k] in FP32
 * (T rounded once to FP32; within every tensor-core precision's bound). The library picks the
 * faster one per (form, degree, cell) for local assembly (measured: the CUDA-core kernel for P1
 * on both cells and for triangles P2, the Burgers forms included; global CSR assembly stays on
 * the tensor cores, batches put the CUDA-core groups in a launch of their own); these flags
 * force one: TENSOR_CORES the tcgen05 kernel, CUDA_CORES the FP32 kernel (ignored where it has
 * no instance). Results of the two differ by rounding, within the precision's bound. */
#define COFFEE_FLAG_TENSOR_CORES 512u
#define COFFEE_FLAG_CUDA_CORES 1024u
/* BURGERS_JAC on the tensor cores with component blocks of at most 128 entries (triangles
 * P1-P3, tetrahedra P1-P2) has two forms: the block form (every component block contracted over
 * [T1 | T2 | T3]) and the factored form, block(ci, cj) = sum_a P[a][cj] V_a^ci + [ci == cj] C
 * with V_a^ci = sum_r u[r][ci] T1[r, a] contracted on the tensor cores and P = |det J| K applied
 * per cell in the epilogue. The factored form is the default for tetrahedra P2 (measured faster
 * there), the block form elsewhere; these flags force one. Results agree within the precision's
 * bound. */
#define COFFEE_FLAG_BURGERS_BLOCKS 2048u
#define COFFEE_FLAG_BURGERS_FACTORED 4096u

/* Number of rows of the element matrix (or length of the element vector): (k+1)(k+2)/2
 * (triangle), (k+1)(k+2)(k+3)/6 (tetrahedron) or (k+1)^2(k+2)/2 (prism), times d for
 * BURGERS_JAC and BURGERS_RESIDUAL. Negative on error. */
int coffee_ndof(int form, int degree, int cell);

/* Reference-element tabulation (section 2, step 2: the static basis tables W, X_D10,
 * X_D01, Y of Listing 1). Host-only, FP64, no CUDA call.
 * Fills a quadrature rule on the reference cell exact for polynomials of degree
 * `quad_degree` (collapsed Gauss-Jacobi product rule) and the degree-`degree`
 * Lagrange basis at its points:
 *   points  [nq][d], weights [nq], basis [nq][ndof], grads [nq][ndof][d]
 *   (grads are derivatives with respect to the reference coordinates).
 * Any output pointer may be NULL; call first with all NULL to query *nq and *ndof.
 * degree 1..6, quad_degree 0..30. */
int coffee_tabulate(int cell, int degree, int quad_degree, int* nq, int* ndof,
                    double* points, double* weights, double* basis, double* grads);

/* Reference tensors of a form (host-only, FP64): T [K][N] with N = ns*ns, where the
 * element matrix (or, for BURGERS_JAC, each of its d*d component blocks) is
 * sum_k G_e[k] T[k] for per-cell geometry/coefficient factors G_e.
 * BURGERS_RESIDUAL returns the BURGERS_JAC tensors (the residual contracts the same ones).
 * Triangles and tetrahedra only: a prism's Jacobian varies over the cell, so it has no
 * reference tensor (COFFEE_ERR_UNSUPPORTED).
 * Pass T = NULL to query *K and *N. */
int coffee_reference_tensor(int form, int degree, int cell, int* K, int* N, double* T);

/* FP64 local assembly (plain one-thread-per-cell kernel), all pointers on the device:
 *   coords    [nverts][d] double
 *   cell2vert [ncells][d+1] int32 (prisms: [ncells][6])
 *   coef      ADVDIFF: [ncoefnodes][1+d] double, row = (eps, b_0, .., b_{d-1})
 *             BURGERS_JAC: u [ncoefnodes][d] double (viscosity nu = 0.01)
 *             MASS/HELMHOLTZ: NULL
 *   cell2dof  ADVDIFF: [ncells][d+1]; BURGERS_JAC: [ncells][ns]; else NULL
 *   out       [ncells][ndof][ndof] double
 * ncoefnodes is not passed here and is taken as unbounded (no validation);
 * coffee_assemble_ex takes the full argument set. ncells == 0 is a no-op.
 * Asynchronous on `stream`; allocates nothing but the first-use table cache. */
int coffee_assemble(int form, int degree, int cell, const double* coords,
                    const int32_t* cell2vert, const double* coef, const int32_t* cell2dof,
                    void* out, int64_t ncells, coffee_stream_t stream);

typedef struct {
  int form;            /* coffee_form */
  int degree;          /* 1..4 */
  int cell;            /* coffee_cell */
  int precision;       /* coffee_precision; FP64 -> double out, else float out */
  double nu;           /* BURGERS_JAC viscosity (0.01 in the benchmarks) */
  const double* coords;      /* device [nverts][d] */
  int64_t nverts;
  const int32_t* cell2vert;  /* device [ncells][d+1] */
  const double* coef;        /* device, layout as in coffee_assemble, or NULL */
  int64_t ncoefnodes;
  const int32_t* cell2dof;   /* device, or NULL */
  void* out;                 /* device [ncells][ndof][ndof], double or float */
  int64_t ncells;
  unsigned flags;            /* COFFEE_FLAG_* */
  /* optional, device [nverts][d][2] float: every coordinate x as a float pair (hi, lo) with
   * hi + lo = x to about 2^-48 |x|, as coffee_split_coords writes them (hi = (float)x and
   * lo = (float)(x - hi) serve as well), or NULL. The tensor-core and CUDA-core kernels on
   * triangles and tetrahedra then take the vertex differences of the Jacobian in FP32
   * ((hi1 - hi0) + (lo1 - lo0)) from the pairs instead of forming them per cell; coords must
   * still be given (badly conditioned cells are recomputed from it in FP64). Ignored by the FP64
   * kernels and by prisms. */
  const float* coords_split;
  /* optional, device, the layout and length of coef in float: every coefficient rounded to
   * nearest ((float)coef[i]), as coffee_round_coef writes it, or NULL. The tensor-core kernels
   * take the coefficients in FP32 either way; given the float copy they read it (half the bytes)
   * instead of converting each coefficient once per cell that uses it, which on this GPU runs on
   * the FP64 pipe. Results are bit for bit those without it. coef must still be given (the FP64
   * kernels read it; every pointer check applies). */
  const float* coef_f32;
  /* entries between the starts of consecutive element matrices in out: 0 (or ndof*ndof) for the
   * contiguous layout [ncells][ndof][ndof]; a larger value pads every matrix, e.g. to a multiple
   * of 32 entries so that each starts on a 128-byte line (element matrices whose size is not a
   * multiple of 32 entries otherwise start at 4- or 8-byte offsets, and warp stores that straddle
   * lines run at about half the rate: tetrahedra P4, 1225 entries). The padding is not written.
   * Local assembly of MASS, HELMHOLTZ and ADVDIFF on triangles and tetrahedra (FP64, tensor-core
   * and CUDA-core kernels); anything else with a nonzero stride other than ndof*ndof returns
   * COFFEE_ERR_INVALID_ARG, as does a stride below ndof*ndof. Ignored by the adjoint entry
   * points. */
  int64_t out_stride;
} coffee_assemble_args;

/* Every coordinate x[i], i < n (n = nverts * d), as a float pair (hi, lo) in split[2i],
 * split[2i+1] with hi + lo = x to 2^-48 |x| (for 2^-100 <= |x| < 2^127, where lo is a normal
 * float): the coords_split input of coffee_assemble_args.
 * For 2^-70 <= |x| < 2^100, hi is x truncated to the 24 significant bits of a float (|hi| <= |x|,
 * same sign) and lo = x - hi rounded to the nearest float; outside that range hi = (float)x and
 * lo = (float)(x - hi); zero gives (0, 0). Device pointers, both 8-byte aligned (else
 * COFFEE_ERR_INVALID_ARG), asynchronous on stream; n == 0 returns COFFEE_OK. */
int coffee_split_coords(const double* coords, int64_t n, float* split, coffee_stream_t stream);

/* Every coefficient coef[i], i < n (n = ncoefnodes * components), rounded to the nearest float:
 * out[i] = (float)coef[i], the coef_f32 input of coffee_assemble_args. One conversion per
 * coefficient node instead of one per cell that reads it (a vertex of a tetrahedral mesh is
 * shared by about 24 cells). Device pointers, asynchronous on stream; n == 0 returns COFFEE_OK. */
int coffee_round_coef(const double* coef, int64_t n, float* out, coffee_stream_t stream);

/* 1 if coffee_assemble_ex has a kernel for (form, degree, cell, precision), else 0.
 * FP64 covers every form, degree 1..4, both cells; the tensor-core precisions cover
 * the combinations whose operands fit in shared memory. Host-only. */
int coffee_supported(int form, int degree, int cell, int precision);

/* The kernel family coffee_assemble_ex runs for local assembly with these arguments and flags:
 * 0 the FP64 kernel, 1 the tensor cores (tcgen05), 2 the FP32 CUDA-core kernel for small
 * element matrices (COFFEE_FLAG_TENSOR_CORES / COFFEE_FLAG_CUDA_CORES); COFFEE_ERR_UNSUPPORTED
 * where coffee_supported is 0. Host-only. */
int coffee_assemble_path(int form, int degree, int cell, int precision, unsigned flags);

/* Local assembly (section 2, Listings 1-2) with a chosen precision. FP64 runs the plain FP64 kernel; the
 * other precisions run the tcgen05 tensor-core contraction with geometry fused into
 * its producer warps (FP32 geometry, FP64 for ill-conditioned cells).
 * Returns COFFEE_ERR_UNSUPPORTED for combinations without a kernel. */
int coffee_assemble_ex(const coffee_assemble_args* a, coffee_stream_t stream);

/* Local assembly (section 2) of data held in HOST memory, where the paper's CPU framework
 * keeps the mesh and the element matrices (section 4): the same kernels as coffee_assemble_ex,
 * with the copies around them. a->coords, a->cell2vert, a->coef, a->cell2dof and a->out are HOST
 * pointers with the layouts of coffee_assemble; out is [ncells][ndof][ndof] (BURGERS_RESIDUAL:
 * [ncells][ndof]), double for FP64 and float otherwise. a->nverts, and a->ncoefnodes for the
 * forms with a coefficient, must be > 0: they size the copies.
 * a->out_stride must be 0 (contiguous results).
 * a->coords_split and a->coef_f32 are ignored: for the tensor-core precisions on triangles and
 * tetrahedra the coordinates are split into (hi, lo) float pairs on the device after their copy,
 * and for every tensor-core precision the coefficients are rounded to floats there.
 * The coordinates and coefficients are copied to the device once; the cells are assembled in
 * `chunks` launches (chunk boundaries on 128-cell tiles), each chunk's inputs copied in and its
 * results copied back on a second, library-owned stream while the next chunk computes.
 * Page-locked host memory lets the copies overlap the kernels; pageable memory works but
 * serialises them. Device staging comes from a library-owned stream-ordered memory pool that
 * keeps its largest size for reuse (coffee_host_pool_trim releases it).
 * Asynchronous: a->out is complete once `stream` has reached the end of this call's work
 * (synchronise `stream`, or wait on an event recorded on it, before reading it).
 * Errors: as coffee_assemble_ex; COFFEE_ERR_INVALID_ARG also for chunks < 1 or a missing size;
 * COFFEE_ERR_NOMEM when the staging buffers cannot be allocated. */
int coffee_assemble_host(const coffee_assemble_args* a, int chunks, coffee_stream_t stream);

/* Releases the device memory the host-buffer pool of the current device holds beyond what
 * pending work still uses. Host-only; returns COFFEE_OK. */
int coffee_host_pool_trim(void);

/* Adjoint of local assembly (new; the paper has no backward pass).
 * Given dout = dL/dA ([ncells][ndof][ndof], double for FP64, float otherwise),
 * ACCUMULATES (+=) dL/dcoords into d_coords [nverts][d] and dL/dcoef into d_coef
 * (coefficient layout; may be NULL when the form has no coefficient). Geometry is
 * recomputed, not stored. The arithmetic runs in the type of dout: FP64, or FP32 for the
 * tensor-core precisions (gradients are always accumulated in FP64). deterministic != 0 sums cell contributions in a fixed
 * order (no floating-point atomics). Device pointers, asynchronous on stream. */
int coffee_assemble_backward(const coffee_assemble_args* a, const void* dout,
                             double* d_coords, double* d_coef, int deterministic,
                             coffee_stream_t stream);

/* Allocation-free deterministic adjoint. The paper has no counterpart: this exists for
 * callers that cannot allocate device memory while they run -- latency-critical loops
 * that must avoid cudaMalloc/cudaFree (they can synchronise the device), applications
 * whose device memory belongs to their own pool or caching allocator, and fixed-budget
 * deployments. It computes exactly what coffee_assemble_backward(a, dout, d_coords,
 * d_coef, deterministic = 1, stream) computes (same kernels, same summation order) but
 * allocates nothing: its scratch is one fixed device array inside the library (about
 * 4.4 MB, reserved on every GPU that loads the library until the process exits).
 *   limits: ncells <= 16384; 1 <= nverts <= 16384; for ADVDIFF with d_coef,
 *           1 <= ncoefnodes <= 16384; forms MASS, HELMHOLTZ, ADVDIFF (BURGERS_JAC returns
 *           COFFEE_ERR_UNSUPPORTED); larger inputs return COFFEE_ERR_INVALID_ARG with a
 *           message naming the limit. COFFEE_FLAG_VALIDATE is rejected: indices must be
 *           in range (check them first with coffee_assemble_backward and the flag).
 *   arguments: as coffee_assemble_backward; d_coords/d_coef are accumulated (+=).
 *   set-up: the first call on a device looks up the array's device address
 *           (cudaGetSymbolAddress) with that device current; make that first call
 *           before any stream capture.
 *   sharing: every call on a device uses the same array and leaves its contents behind;
 *           each call clears what must start at zero. Calls that overlap on the GPU
 *           (other streams, other host threads) race on the array: serialise them.
 *   errors: device-side index errors set an error word in the same array; it keeps them
 *           until coffee_check_errors reads it (with the library's own word) and clears it.
 *           The reference tensor is copied into the array only when the previous call on the
 *           device used another (form, degree, cell). */
int coffee_assemble_backward_noalloc(const coffee_assemble_args* a, const void* dout,
                                     double* d_coords, double* d_coef, coffee_stream_t stream);

/* Mixed batch: several (form, degree, cell) groups assembled by one persistent tensor-core
 * launch (the paper runs one specialised kernel per form, degree and cell shape, sections 4-5),
 * plus one launch of the CUDA-core kernel for the groups of small element matrices that run
 * there by default (P1 simplices and P2 triangles; coffee_assemble_path), unless groups[0].flags
 * has COFFEE_FLAG_TENSOR_CORES, which keeps every group on the tensor cores.
 * Each group is a coffee_assemble_args (its own inputs, output and cell count); all groups
 * share one tensor-core precision and are MASS, HELMHOLTZ or ADVDIFF. The plan (host)
 * uploads the groups' tables, cuts every tensor-core group into 128-cell tiles and gives each
 * CTA a contiguous range of tiles of about equal cost (bytes written + item_overhead per
 * 128-output slice), and numbers the CUDA-core groups' 32-cell warp tiles across the groups.
 * Planning allocates device memory and synchronises; launching only enqueues the (at most two)
 * kernels, so it can be captured in a CUDA graph. The plan refers to the groups' device
 * buffers, which must stay valid while it is launched. Every group's result equals, bit for
 * bit, its own coffee_assemble_ex on the same kernel family.
 *   grid <= 0 selects one CTA per SM; item_overhead < 0 selects the default (16384). */
int coffee_batch_plan(const coffee_assemble_args* groups, int ngroups, int grid, double item_overhead,
                      void** plan);
/* The same plan with a measured cost per group instead of the byte model:
 *   tile_cost  host [ngroups], the cost of one full 128-cell tile of group i in any unit
 *              (e.g. its measured time); a ragged tile costs cells/128 of it. Every entry must
 *              be positive and finite, else COFFEE_ERR_INVALID_ARG. Not retained. */
int coffee_batch_plan_costs(const coffee_assemble_args* groups, int ngroups, int grid, const double* tile_cost,
                            void** plan);
int coffee_batch_launch(void* plan, coffee_stream_t stream);
void coffee_batch_free(void* plan);
/* The split both planners use (host-only, no CUDA call): `items` work items with costs
 * cost[i] >= 0 (finite) go to `grid` CTAs in contiguous ranges; CTA b takes items
 * [ranges[b], ranges[b+1]), with ranges[0] = 0, ranges[grid] = items, and the cut after CTA b
 * placed at the first item where the running cost reaches (b+1)/grid of the total.
 *   cost host [items]; ranges host [grid+1], out. COFFEE_ERR_INVALID_ARG for items < 0,
 *   grid < 1, NULL pointers or a negative or non-finite cost. */
int coffee_batch_split(const double* cost, int64_t items, int grid, int64_t* ranges);

/* ---- Global assembly: the consumer of local assembly ----
 * Local assembly yields each cell's contribution to the global linear system (section 2);
 * the framework that runs the paper's kernels over all cells of the mesh (section 4) adds
 * these element matrices into a global sparse matrix through each cell's local-to-global
 * dof map. These entry points do that step on the GPU in CSR form. Rows and columns share
 * the map (the forms are square):
 *   l2g [ncells][nloc] int32, global row of each row of the element matrix, in [0, nrows).
 *   For scalar forms nloc = ns and l2g is the cell-to-node map of the degree-k space; for
 *   BURGERS_JAC nloc = d*ns, component-blocked like the element matrix
 *   (l2g[e][c*ns + i] = global dof of component c at node i). */

/* CSR sparsity of the global matrix: (r, c) is stored iff some cell e has r = l2g[e][i] and
 * c = l2g[e][j]; the columns of each row ascend.
 *   rowptr  device [nrows+1] int64;  colidx  device [nnz] int32;  nnz  host.
 * Two calls. With colidx == NULL the call writes rowptr and *nnz; then, with colidx
 * allocated for nnz entries and the same rowptr, it writes the columns. Both calls allocate
 * their scratch on the stream (cudaMallocAsync) and synchronise it before returning, so
 * errors are reported by the call itself: COFFEE_ERR_INVALID_ARG for an l2g entry outside
 * [0, nrows) or a rowptr that does not match l2g, COFFEE_ERR_UNSUPPORTED when a row
 * gathers more than 4096 entries before deduplication (the sum of nloc over the cells that
 * contain its dof). Limits: 1 <= nloc <= 128; ncells, nrows <= 2^31 - 1. */
int coffee_sparsity(const int32_t* l2g, int64_t ncells, int nloc, int64_t nrows, int64_t* rowptr,
                    int32_t* colidx, int64_t* nnz, coffee_stream_t stream);

/* Position of every element-matrix entry in the CSR arrays:
 * map[e][i*nloc + j] = k such that colidx[k] == l2g[e][j], rowptr[l2g[e][i]] <= k < rowptr[l2g[e][i]+1].
 *   map  device uint32, 16-byte aligned, nnz below 2^32, stored in the blocks the fused assembly
 *        reads: with npad = nloc*nloc rounded up to a multiple of 4, cells are grouped by 32
 *        (ncells padded up to a multiple of 32) and entries by 32; block (cb, ob) holds
 *        [32 cells][w] values, w = min(32, npad - 32*ob), at offset 32*(cb*npad + 32*ob), so
 *        entry (e, idx) is at 32*((e/32)*npad + 32*(idx/32)) + (e%32)*w + idx%32. Length
 *        ceil(ncells/32)*32*npad; padding entries are 0xffffffff.
 * Asynchronous; an entry that cannot be found (l2g and the pattern disagree) is set to
 * 0xffffffff and raises COFFEE_ERR_DEVICE_INDEX in coffee_check_errors. */
int coffee_csr_map(const int32_t* l2g, int64_t ncells, int nloc, const int64_t* rowptr, const int32_t* colidx,
                   int64_t nrows, uint32_t* map, coffee_stream_t stream);

/* Fused global assembly: vals[map[e][o]] += A_e[o] for every cell e and entry o, where A_e
 * is the element matrix coffee_assemble_ex computes for *a (a->out is ignored). The tensor-core
 * precisions add the entries straight from the accumulators (the element matrices are never
 * written to memory) into float vals; FP64 adds into double vals.
 *   vals  device [nnz], float (tensor-core precisions) or double (FP64); the call ADDS into it,
 *         so zero it first for a new matrix.
 * Entries are added with floating-point atomics: the order in which the contributions to one
 * global entry are summed is not fixed. A map entry >= nnz is skipped and raises
 * COFFEE_ERR_DEVICE_INDEX in coffee_check_errors. The tensor-core path covers MASS, HELMHOLTZ
 * and ADVDIFF (coffee_supported combinations whose operands stay resident in shared memory);
 * FP64 covers every form. Otherwise COFFEE_ERR_UNSUPPORTED. */
int coffee_assemble_csr(const coffee_assemble_args* a, const uint32_t* map, void* vals, int64_t nnz,
                        coffee_stream_t stream);

/* 1 if coffee_assemble_csr has a kernel for (form, degree, cell, precision), else 0. Host-only. */
int coffee_csr_supported(int form, int degree, int cell, int precision);

/* Device error word: synchronises `stream`, returns COFFEE_ERR_DEVICE_INDEX if a
 * validated launch met an out-of-range index, COFFEE_ERR_TIMEOUT if a kernel wait
 * gave up, COFFEE_OK otherwise, and clears the word. */
int coffee_check_errors(coffee_stream_t stream);

/* Message of the last failing call on this thread ("" if none). */
const char* coffee_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* COFFEE_H */
