// ps_loads.cuh -- pressure loads on the mass points of the wing (Sec. 4.1,
// fluid-to-solid coupling paragraph): the static pressure interpolated to
// every node with a smoothed discrete delta function, and per triangle the
// force -p_v (A/3) n on each of its vertices.
//
// Kernel (the paper cites a smoothing technique for discrete delta functions
// without printing one; reading): the 4-point cosine kernel
// phi(r) = (1/4)(1 + cos(pi r/2)), |r| <= 2, convolved with the unit box,
//   phi_s(r) = (1/4)(1 + (2/pi)(sin(pi(r+1/2)/2) - sin(pi(r-1/2)/2))), |r| <= 3/2,
//   phi_s(r) = (1/4)((5/2 - |r|) - (2/pi) sin(pi(|r|-1/2)/2)),        3/2 < |r| < 5/2,
// zero beyond; five grid points per axis, periodic grid. All sums in double.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ps {

struct LoadArgs {
    int n, nz;            // grid n x n x nz, spacing dx on every axis
    double dx;
    const double* xw;     // n_nodes x 3, wing frame
    int n_nodes;
    const int32_t* tri;   // n_tri x 3
    int n_tri;
    double R[9], XO[3];   // wing frame -> global
};

__device__ __forceinline__ double delta_smoothed(double r) {
    r = fabs(r);
    const double c = 2.0 / M_PI, h = 0.5 * M_PI;
    if (r <= 1.5) return 0.25 * (1.0 + c * (sin(h * (r + 0.5)) - sin(h * (r - 0.5))));
    if (r < 2.5) return 0.25 * ((2.5 - r) - c * sin(h * (r - 0.5)));
    return 0.0;
}

__device__ __forceinline__ void global_node(const LoadArgs& a, int v, double X[3]) {
    const double* x = a.xw + 3 * v;
    for (int r = 0; r < 3; ++r) X[r] = a.XO[r] + a.R[3 * r] * x[0] + a.R[3 * r + 1] * x[1] + a.R[3 * r + 2] * x[2];
}

// One thread per node: p at the node from the 6 x 6 x 6 grid points around it.
template <typename T>
__global__ void k_node_pressure(LoadArgs a, const T* __restrict__ pf, double* __restrict__ pn) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.n_nodes) return;
    double X[3];
    global_node(a, v, X);
    int lo[3];
    double w[3][6];
    for (int r = 0; r < 3; ++r) {
        const double g = X[r] / a.dx;
        lo[r] = (int)floor(g) - 2;
        for (int q = 0; q < 6; ++q) w[r][q] = delta_smoothed(g - (double)(lo[r] + q));
    }
    const long n = a.n, nz = a.nz;
    double acc = 0.0;
    for (int i = 0; i < 6; ++i) {
        const long xi = (((long)lo[0] + i) % n + n) % n;
        for (int j = 0; j < 6; ++j) {
            const long yj = (((long)lo[1] + j) % n + n) % n;
            const double wij = w[0][i] * w[1][j];
            const T* row = pf + (xi * n + yj) * nz;
            double s = 0.0;
            for (int k = 0; k < 6; ++k) s += w[2][k] * (double)row[(((long)lo[2] + k) % nz + nz) % nz];
            acc += wij * s;
        }
    }
    pn[v] = acc;
}

// One warp per node: F_v = -p_v sum over the triangles containing v of
// ((b - a) x (c - a)) / 6 (global frame); the lanes scan the triangles in
// strided index order and combine by a fixed shuffle tree (deterministic).
__global__ void k_node_loads(LoadArgs a, const double* __restrict__ pn, double* __restrict__ F) {
    const int v = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (v >= a.n_nodes) return;   // whole warps leave together
    double s[3] = {0.0, 0.0, 0.0};
    for (int t = lane; t < a.n_tri; t += 32) {
        const int i0 = a.tri[3 * t], i1 = a.tri[3 * t + 1], i2 = a.tri[3 * t + 2];
        if (i0 != v && i1 != v && i2 != v) continue;
        double A[3], B[3], C[3];
        global_node(a, i0, A);
        global_node(a, i1, B);
        global_node(a, i2, C);
        const double e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        const double e2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
        s[0] += e1[1] * e2[2] - e1[2] * e2[1];
        s[1] += e1[2] * e2[0] - e1[0] * e2[2];
        s[2] += e1[0] * e2[1] - e1[1] * e2[0];
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int r = 0; r < 3; ++r) s[r] += __shfl_down_sync(0xffffffffu, s[r], o);
    if (lane == 0) {
        const double f = -pn[v] / 6.0;
        for (int r = 0; r < 3; ++r) F[3 * v + r] = f * s[r];
    }
}

}  // namespace ps
