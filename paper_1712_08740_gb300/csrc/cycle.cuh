// Device-resident state of the restarted FGMRES recurrences, one entry per
// right-hand side (see cycle.cu).
#pragma once

#include <cuda_runtime.h>

namespace helm {

enum RhsStatus { ST_LIVE = 0, ST_CONVERGED = 1, ST_MAXIT = 2, ST_BROKE = 3 };

struct CycleState {
    int m;                 // restart length
    double2 *R;            // [nrhs][(m+1) x m] rotated Hessenberg, column-major
    double2 *g;            // [nrhs][m+1] rotated right-hand side of the least-squares problem
    double *cs;            // [nrhs][m] Givens cosines
    double2 *sn;           // [nrhs][m] Givens sines
    double2 *Q;            // [nrhs][(m+1) x (m+1)] product of the rotations, column-major
    double *fnorm;         // [nrhs] ||f||
    double *beta;          // [nrhs] ||r|| at the start of the cycle
    double *relres;        // [nrhs] last true relative residual
    int *k;                // [nrhs] steps taken in the current cycle
    int *its;              // [nrhs] steps taken in total
    int *status;           // [nrhs] RhsStatus
    int *act_it;           // [nrhs] 1 while the right-hand side takes Arnoldi steps
    int *act_cy;           // [nrhs] 1 while it is part of the current cycle
    int *any_dev;          // [1] scratch for the cross-block "any active" flag (zero at rest)
    unsigned *ticket;      // [1] ticket of the least-squares blocks (zero at rest)
};

void prepare_cycle_kernels();   // shared-memory attributes; call outside graph capture

void launch_cycle_init(const CycleState &S, const double *nrm2, int nrhs, int *host_flag,
                       cudaStream_t st);
// least-squares update of step j and v_{j+1} = w / ||w|| in one launch;
// SV: basis type (double2, or float4 for the double-single basis). The
// scaling of a right-hand side that stops at this step may be skipped (its
// v_{j+1} is never read again by FGMRES); w = nullptr launches the
// least-squares part only, for a caller that scales w itself.
template <typename SV>
void launch_givens_scale(const CycleState &S, int j, const double2 *hb, int hstride, int two,
                         const double *nrm2, int nrhs, double tol, int max_iters, int *host_flag,
                         SV *w, size_t sw, size_t N, cudaStream_t st);
void launch_backsolve(const CycleState &S, double2 *y, int nrhs, cudaStream_t st);
void launch_cycle_check(const CycleState &S, const double *nrm2, int nrhs, double tol,
                        int max_iters, int *host_flag, cudaStream_t st);

}  // namespace helm
