// Droplet shape from its second moments: 3x3 symmetric eigen-decomposition
// and the deformation D of Sec. 2, Eq. 4.  Shared by the single-box and the
// batched reductions.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

namespace lbmgb {
namespace {

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations.  a is
// overwritten; on return lam holds the eigenvalues and v the eigenvectors
// (column k of v belongs to lam[k]).
__device__ void jacobi3(double a[3][3], double lam[3], double v[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) v[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        const double off = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
        const double scale = fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2]);
        if (off <= 1e-300 || off <= 1e-17 * scale) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (a[p][q] == 0.0) continue;
                // rotation angle that annihilates a[p][q]
                const double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) {  // A <- A J
                    const double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - s * akq;
                    a[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {  // A <- J^T A
                    const double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - s * aqk;
                    a[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {  // V <- V J
                    const double vkp = v[k][p], vkq = v[k][q];
                    v[k][p] = c * vkp - s * vkq;
                    v[k][q] = s * vkp + c * vkq;
                }
            }
    }
    for (int k = 0; k < 3; ++k) lam[k] = a[k][k];
}

// From the ten moments m: the moments, D, axes (axes[3*a + k]), eigenvalues
// and centre of mass into result[0..25] (the layout of lbm_deformation).
__device__ void deformation_from_moments(const double (&m)[10], double* __restrict__ result) {
    for (int k = 0; k < 10; ++k) result[k] = m[k];
    const double mass = m[0];
    const double c[3] = {m[1] / mass, m[2] / mass, m[3] / mass};
    double I[3][3];
    I[0][0] = m[4] / mass - c[0] * c[0];
    I[0][1] = I[1][0] = m[5] / mass - c[0] * c[1];
    I[0][2] = I[2][0] = m[6] / mass - c[0] * c[2];
    I[1][1] = m[7] / mass - c[1] * c[1];
    I[1][2] = I[2][1] = m[8] / mass - c[1] * c[2];
    I[2][2] = m[9] / mass - c[2] * c[2];
    double lam[3], v[3][3];
    jacobi3(I, lam, v);
    // order by decreasing eigenvalue
    int ord[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (lam[ord[j]] > lam[ord[i]]) { const int tmp = ord[i]; ord[i] = ord[j]; ord[j] = tmp; }
    for (int k = 0; k < 3; ++k) {
        const int col = ord[k];
        int big = 0;
        for (int a = 1; a < 3; ++a)
            if (fabs(v[a][col]) > fabs(v[big][col])) big = a;
        const double sgn = v[big][col] < 0.0 ? -1.0 : 1.0;
        for (int a = 0; a < 3; ++a) result[11 + 3 * a + k] = sgn * v[a][col];
        result[20 + k] = lam[col];
        result[23 + k] = c[k];
    }
    const double a1 = sqrt(fmax(lam[ord[0]], 0.0)), a3 = sqrt(fmax(lam[ord[2]], 0.0));
    result[10] = (a1 - a3) / (a1 + a3);
}

}  // namespace
}  // namespace lbmgb
