/* Float64 gradient-check library (libbp1104_f64.so): the double
 * instantiations of the library's direct backprojection and direct adjoint
 * kernels (templates on the scalar type, bp_direct.cuh).  TEST SUPPORT ONLY:
 * the product library computes in float32 (Sect. 3.1's single precision) and
 * uses float64 on the GPU only to build and invert projection matrices.  In
 * float64 a finite-difference check of the backprojection against its
 * transpose (torch.autograd.gradcheck with its default step and tolerances)
 * is exact to about 1e-10, which float32 arithmetic cannot give.
 *
 * Both entry points follow Sect. 3.1, Listing 1 (and its transpose): for
 * every voxel x of the L x L x L volume (voxel size R mm, centre of voxel
 * (0,0,0) at O mm, x fastest) and projection i, (uw, vw, w) = A_i (x, 1),
 * u = uw / w, v = vw / w, bilinear weights of the four pixels around
 * (u, v), zero outside the detector (Sect. 3.3), weight 1 / w^2.
 *
 * Arguments: images and vol are DEVICE pointers (float64, caller-owned);
 * images: n x isy x isx row-major; A: HOST pointer to n row-major 3x4
 * float64 matrices.  stream: a cudaStream_t (NULL: the legacy default
 * stream); both calls are asynchronous on it.  Errors: BP_EINVAL for bad
 * sizes or NULL pointers, BP_ECUDA for a CUDA error; the message is
 * available from bp_f64_last_error() on the calling thread. */
#ifndef BP1104_F64_H
#define BP1104_F64_H

#include "bp1104.h"

#ifdef __cplusplus
extern "C" {
#endif

/* vol += B images: the backprojection (Sect. 3.1, Listing 1). */
bp_status bp_f64_backproject(int L, double R, const double O[3], int isx, int isy, const double *images,
                             const double *A, int n, double *vol, void *stream);

/* images += B^T vol: the transpose, a voxel-driven forward projection with
 * atomic scatter of f(x) / w^2 times the four bilinear weights. */
bp_status bp_f64_adjoint(int L, double R, const double O[3], int isx, int isy, const double *vol,
                         const double *A, int n, double *images, void *stream);

/* Text of the calling thread's last error. */
const char *bp_f64_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
