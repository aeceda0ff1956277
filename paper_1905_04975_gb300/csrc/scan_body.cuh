// Device helpers shared by the scan kernels and the server kernel.
#pragma once

#include "common.cuh"

namespace gbr {

// Eigenvalue at diagonal position i of a standard real Schur form (Eq. 4):
// a 1x1 block s gives (s, 0); a standardized 2x2 block [[a, b], [c, a]] gives
// a + i sqrt(-bc) on its first row and a - i sqrt(-bc) on its second.
__device__ __forceinline__ void eig_at(int n, const double* __restrict__ S, int ldS, int i,
                                       double* re, double* im) {
    *re = __ldcg(&S[cm(i, i, ldS)]);
    *im = 0.0;
    if (i + 1 < n && __ldcg(&S[cm(i + 1, i, ldS)]) != 0.0) {
        *im = sqrt(fabs(__ldcg(&S[cm(i, i + 1, ldS)]))) * sqrt(fabs(__ldcg(&S[cm(i + 1, i, ldS)])));
    } else if (i > 0 && __ldcg(&S[cm(i, i - 1, ldS)]) != 0.0) {
        *im = -(sqrt(fabs(__ldcg(&S[cm(i - 1, i, ldS)]))) * sqrt(fabs(__ldcg(&S[cm(i, i - 1, ldS)]))));
    }
}

}  // namespace gbr
