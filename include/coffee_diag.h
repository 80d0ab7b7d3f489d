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

#ifdef __cplusplus
}
#endif

#endif /* COFFEE_DIAG_H */
