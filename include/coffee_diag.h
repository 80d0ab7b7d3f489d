/* Diagnostics of libcoffee.so: exercise the library's failure reporting on a real device
 * without faulting or hanging it.
 *
 * Every wait inside the library's kernels (mbarrier hand-offs between producer, MMA and
 * epilogue roles) is bounded: after about 4e9 SM cycles (~2 s) it sets COFFEE_ERR_TIMEOUT in
 * the device error word and the kernel unwinds (releasing its tensor memory), so the context
 * stays usable and coffee_check_errors() reports the failure. */
#ifndef COFFEE_DIAG_H
#define COFFEE_DIAG_H

#include "coffee.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Enqueues on `stream` one thread that waits, through the same bounded wait, on an mbarrier
 * that nothing arrives at. It gives up after the bound and returns; the next
 * coffee_check_errors(stream) returns COFFEE_ERR_TIMEOUT (and clears the word). Returns
 * COFFEE_OK once enqueued, COFFEE_ERR_CUDA on a launch error. */
int coffee_diag_wait_timeout(coffee_stream_t stream);

/* The tensor-core operand image of a form's reference tensors, byte for byte as the library
 * uploads it (host-only, no CUDA call; for inspection and tests). Triangles and tetrahedra:
 * for each M-tile of 128 outputs, the hi part and, for split precisions, the lo part, each
 * 128 rows (outputs) x kbytes bytes (K columns of tf32 or bf16) in the no-swizzle K-major
 * canonical layout of the tcgen05 shared-memory descriptors: byte kb of row r of a part is at
 *   (r / 8) * 8 * kbytes + (kb / 16) * 128 + (r % 8) * 16 + kb % 16
 * (core matrices of 8 rows x 16 bytes, 128 bytes apart along K, 8 * kbytes apart down the
 * rows). Where meta[5] (exact A) is 1 a tile holds one part of integers and the float scale of
 * every column follows the tiles at byte meta[7]. Prisms use their own streamed layout.
 *   img     host, out, or NULL to query the size;  nbytes  host, out: the image's size;
 *   meta    host [8], out, or NULL: mtiles, kbytes, kelems (padded K), K, parts, aexact,
 *           ksteps_off (Burgers), scale_off.
 * COFFEE_ERR_UNSUPPORTED for FP64 or a combination without a tensor-core kernel. */
int coffee_table_image(int form, int degree, int cell, int precision, uint8_t* img, int64_t* nbytes,
                       int64_t* meta);

#ifdef __cplusplus
}
#endif

#endif /* COFFEE_DIAG_H */
