// ps_adjoint.cuh -- discrete adjoint of one time step and of the wing mask
// rasteriser (no counterpart in the paper; the exact transpose of the step's
// operations, for objectives J = sum_n (a_n . F^n + b_n . M^n)).
//
// Conventions: U holds Fourier coefficients c (u = inverse(c), no scaling;
// forward(u) = DFT(u) / n^3). Adjoint variables live on the same compact
// spectral layout with the inner product Re sum w conj(x) y (w = 1 on the
// kz = 0 plane, 2 elsewhere), under which inverse* = n^3 forward and
// forward* = inverse / n^3; truncation, projection, E and i k x are
// self-adjoint mode by mode. Per reversed step n (lam = dL/du^{n+1},
// mu = dL/dH^{n+1}):
//   Gbar = a1 lam + mu  (a1 = 1.5 dt E, or dt E for the Euler start step)
//   G    = P Gbar        -> nbar = inverse(G) / n^3       (physical)
//   lam' = E lam,  mu' = -0.5 dt E^2 lam  (0 for the start step)
//   ubar = omega x nbar - (chi/eta) nbar + (dx^3/eta) chi (a + b x r)
//   wbar = nbar x u
//   dJ/dchi = -(1/eta) nbar . (u - us) + (dx^3/eta) (a + b x r) . (u - us)
//   dJ/dus  = (chi/eta) nbar - (dx^3/eta) chi (a + b x r)
//   lam' += n^3 [forward(ubar) + i k x forward(wbar)]
#pragma once
#include "ps_kernels.cuh"

namespace ps {

struct AdjW {
    double a[3], b[3];   // dJ/dF, dJ/dM of this step
    int first;           // reversing the integrating-factor Euler start step
};

// Spectral part 1: G = P (a1 lam + mu); lam <- E lam; mu <- -0.5 dt E^2 lam.
template <typename T>
__global__ void k_adj_spec1(KP kp, cplx<T>* __restrict__ lam, cplx<T>* __restrict__ mu, cplx<T>* __restrict__ G,
                            const T* __restrict__ Ex, const T* __restrict__ Ez, int first) {
    using C2 = cplx<T>;
    const int K = kp.K, Kz = kp.Kz, Kzp = kp.Kzp, mm = kp.mmax;
    const size_t FS = (size_t)K * K * Kzp;
    const size_t tot = (size_t)K * K * Kz;
    const T dt = (T)kp.dt, s = (T)kp.ks, sz = (T)kp.ksz;
    // 32-bit index arithmetic: K^2 Kz < 2^27 for every grid the library builds
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (uint32_t)tot; i += gridDim.x * blockDim.x) {
        const int cz = (int)(i % (uint32_t)Kz);
        const uint32_t r = i / (uint32_t)Kz;
        const int cx = (int)(r % (uint32_t)K), cy = (int)(r / (uint32_t)K);
        const size_t o = ((size_t)cy * K + cx) * Kzp + cz;
        const T E = Ex[cx] * Ex[cy] * Ez[cz];
        const T a1 = first ? dt * E : (T)1.5 * dt * E;
        const T a2 = first ? (T)0 : (T)0.5 * dt * E * E;
        C2 g[3], l[3];
        for (int f = 0; f < 3; ++f) {
            l[f] = lam[f * FS + o];
            const C2 m = mu[f * FS + o];
            g[f] = cmk<C2>(a1 * l[f].x + m.x, a1 * l[f].y + m.y);
        }
        const int mx = cmode_of(cx, mm, K), my = cmode_of(cy, mm, K);
        const T kx = s * (T)mx, ky = s * (T)my, kz = sz * (T)cz;
        if (mx == 0 && my == 0 && cz == 0) {
            if (!kp.mean_free) g[0] = g[1] = g[2] = cmk<C2>((T)0, (T)0);
        } else {
            const T ik2 = (T)1 / (kx * kx + ky * ky + kz * kz);
            const T dr = (kx * g[0].x + ky * g[1].x + kz * g[2].x) * ik2;
            const T di = (kx * g[0].y + ky * g[1].y + kz * g[2].y) * ik2;
            g[0].x -= kx * dr; g[0].y -= kx * di;
            g[1].x -= ky * dr; g[1].y -= ky * di;
            g[2].x -= kz * dr; g[2].y -= kz * di;
        }
        for (int f = 0; f < 3; ++f) {
            G[f * FS + o] = g[f];
            lam[f * FS + o] = cmk<C2>(E * l[f].x, E * l[f].y);
            mu[f * FS + o] = cmk<C2>(-a2 * l[f].x, -a2 * l[f].y);
        }
    }
}

// lam += n^3 (Ub + i k x Wb).
template <typename T>
__global__ void k_adj_spec2(KP kp, cplx<T>* __restrict__ lam, const cplx<T>* __restrict__ Ub,
                            const cplx<T>* __restrict__ Wb) {
    using C2 = cplx<T>;
    const int K = kp.K, Kz = kp.Kz, Kzp = kp.Kzp, mm = kp.mmax;
    const size_t FS = (size_t)K * K * Kzp;
    const size_t tot = (size_t)K * K * Kz;
    const T s = (T)kp.ks, sz = (T)kp.ksz;
    const T n3 = (T)(1.0 / kp.invn3);
    // 32-bit index arithmetic: K^2 Kz < 2^27 for every grid the library builds
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (uint32_t)tot; i += gridDim.x * blockDim.x) {
        const int cz = (int)(i % (uint32_t)Kz);
        const uint32_t r = i / (uint32_t)Kz;
        const int cx = (int)(r % (uint32_t)K), cy = (int)(r / (uint32_t)K);
        const size_t o = ((size_t)cy * K + cx) * Kzp + cz;
        const T kx = s * (T)cmode_of(cx, mm, K), ky = s * (T)cmode_of(cy, mm, K), kz = sz * (T)cz;
        const C2 wx = Wb[o], wy = Wb[FS + o], wz = Wb[2 * FS + o];
        const C2 c0 = cmk<C2>(ky * wz.x - kz * wy.x, ky * wz.y - kz * wy.y);
        const C2 c1 = cmk<C2>(kz * wx.x - kx * wz.x, kz * wx.y - kx * wz.y);
        const C2 c2 = cmk<C2>(kx * wy.x - ky * wx.x, kx * wy.y - ky * wx.y);
        const C2 cc[3] = {cmk<C2>(-c0.y, c0.x), cmk<C2>(-c1.y, c1.x), cmk<C2>(-c2.y, c2.x)};
        for (int f = 0; f < 3; ++f) {
            const C2 u = Ub[f * FS + o];
            const C2 l = lam[f * FS + o];
            lam[f * FS + o] = cmk<C2>(l.x + n3 * (u.x + cc[f].x), l.y + n3 * (u.y + cc[f].y));
        }
    }
}

// Physical pointwise adjoint. u, w: velocity and vorticity of the step (3 x
// n^3 each), overwritten by ubar and wbar; nb: inverse(G) (scaled here by
// 1/n^3). Writes dJ/dchi and dJ/dus of this step.
// Memory bound: the thirteen loads of a point are issued before its
// arithmetic, with a register budget (four blocks of 256 threads per SM) that
// keeps them all in flight.
template <typename T>
__global__ void __launch_bounds__(256, 4) k_adj_point(KP kp, AdjW aw, T* __restrict__ u, T* __restrict__ w, const T* __restrict__ nb,
                            const T* __restrict__ chi, const T* __restrict__ us, T* __restrict__ gchi,
                            T* __restrict__ gus) {
    const int n = kp.n, nz = kp.nz;
    const size_t n3 = (size_t)n * n * nz;
    // constants in T: no double arithmetic and no 64-bit division per point
    const T inv_eta = (T)kp.inv_eta, invn3 = (T)kp.invn3, dx = (T)kp.dx;
    const T f = (T)(kp.dx * kp.dx * kp.dx * kp.inv_eta);
    const T x0 = (T)kp.x0[0], y0 = (T)kp.x0[1], z0 = (T)kp.x0[2];
    const T a0 = (T)aw.a[0], a1 = (T)aw.a[1], a2 = (T)aw.a[2];
    const T b0 = (T)aw.b[0], b1 = (T)aw.b[1], b2 = (T)aw.b[2];
    // 32-bit point index (n^3 < 2^32 for every built grid size)
    const uint32_t n3u = (uint32_t)n3, un = (uint32_t)n, unz = (uint32_t)nz;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n3u; p += gridDim.x * blockDim.x) {
        {
            const uint32_t q = p / unz, k = p - q * unz;
            const uint32_t i = q / un, j = q - i * un;
            const T nbx0 = nb[p], nby0 = nb[n3 + p], nbz0 = nb[2 * n3 + p];
            const T ux = u[p], uy = u[n3 + p], uz = u[2 * n3 + p];
            const T wx = w[p], wy = w[n3 + p], wz = w[2 * n3 + p];
            const T c = chi[p];
            const T sx = us[p], sy = us[n3 + p], sz = us[2 * n3 + p];
            const T rx = (T)i * dx - x0, ry = (T)j * dx - y0;
            const T nbx = nbx0 * invn3, nby = nby0 * invn3, nbz = nbz0 * invn3;
            const T ce = c * inv_eta;
            // ubar = w x nbar - c nbar ; wbar = nbar x u
            T bx = wy * nbz - wz * nby - ce * nbx;
            T by = wz * nbx - wx * nbz - ce * nby;
            T bz = wx * nby - wy * nbx - ce * nbz;
            const T vx = nby * uz - nbz * uy;
            const T vy = nbz * ux - nbx * uz;
            const T vz = nbx * uy - nby * ux;
            // dJ/dchi is needed at every cell (also where chi = 0); the force
            // and moment term uses dJ/dp = a + b x r, p = chi (u - us)
            const T dx_ = ux - sx, dy_ = uy - sy, dz_ = uz - sz;
            const T rz = (T)k * dx - z0;
            const T gx = a0 + b1 * rz - b2 * ry;
            const T gy = a1 + b2 * rx - b0 * rz;
            const T gz = a2 + b0 * ry - b1 * rx;
            const T cf = f * c;
            bx += cf * gx; by += cf * gy; bz += cf * gz;
            const T gc = -inv_eta * (nbx * dx_ + nby * dy_ + nbz * dz_) + f * (gx * dx_ + gy * dy_ + gz * dz_);
            const T gsx = ce * nbx - cf * gx, gsy = ce * nby - cf * gy, gsz = ce * nbz - cf * gz;
            u[p] = bx; u[n3 + p] = by; u[2 * n3 + p] = bz;
            w[p] = vx; w[n3 + p] = vy; w[2 * n3 + p] = vz;
            gchi[p] = gc;
            gus[p] = gsx; gus[n3 + p] = gsy; gus[2 * n3 + p] = gsz;
        }
    }
}

// ------------------------------------------------ rasteriser VJP
__device__ __forceinline__ double chi_profile_d(double d, double tw, double h, int profile) {
    if (profile == 1) {
        const double t = tanh((d - tw) / h);
        return -0.5 * (1.0 - t * t) / h;
    }
    if (d <= tw - h || d >= tw + h) return 0.0;
    return -0.25 * M_PI / h * sin(M_PI * (d - tw + h) / (2.0 * h));
}

// One grid point p with closest triangle t: dJ/dX (global vertex positions)
// accumulated into gX with atomics. The closest triangle is held fixed; the
// distance derivative is -beta_v (p - q)/delta (envelope theorem), the
// barycentric weights are differentiated on their active face.
template <typename T>
__device__ void vjp_point(const MaskWs& m, const MaskArgs& a, uint32_t p, int t, const T* __restrict__ gchi,
                          const T* __restrict__ gus, const T* __restrict__ chi, double* __restrict__ gX) {
    const size_t n = a.n, nz = a.nz, n3 = n * n * nz;
    const int k = (int)(p % nz), j = (int)((p / nz) % n), i = (int)(p / (n * nz));
    const double P[3] = {i * a.dx, j * a.dx, k * a.dx};
    const int id[3] = {a.tri[3 * t], a.tri[3 * t + 1], a.tri[3 * t + 2]};
    double X[3][3];
    for (int v = 0; v < 3; ++v)
        for (int r = 0; r < 3; ++r) X[v][r] = m.xg[3 * id[v] + r];
    double Pr[3], V[3][3];
    for (int r = 0; r < 3; ++r) {
        Pr[r] = P[r] - X[0][r];
        V[0][r] = 0.0;
        V[1][r] = X[1][r] - X[0][r];
        V[2][r] = X[2][r] - X[0][r];
    }
    double beta[3];
    const double d = sqrt(closest_tri<double>(Pr, V[0], V[1], V[2], beta));
    double q[3];
    for (int r = 0; r < 3; ++r) q[r] = beta[0] * X[0][r] + beta[1] * X[1][r] + beta[2] * X[2][r];
    double acc[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    const double cb = (double)gchi[p];
    if (d > 0.0 && cb != 0.0) {
        const double gd = cb * chi_profile_d(d, a.tw, a.h, a.profile);
        for (int v = 0; v < 3; ++v)
            for (int r = 0; r < 3; ++r) acc[v][r] += gd * (-beta[v] * (P[r] - q[r]) / d);
    }
    const bool has_us = (a.profile == 1) || (double)chi[p] > 0.0;
    if (has_us) {
        const double ub[3] = {(double)gus[p], (double)gus[n3 + p], (double)gus[2 * n3 + p]};
        double g[3];
        for (int v = 0; v < 3; ++v) {   // dJ/dbeta_v = ub . (R vw_v)
            double s = 0.0;
            for (int r = 0; r < 3; ++r) {
                double rv = 0.0;
                for (int c = 0; c < 3; ++c) rv += a.R[3 * r + c] * a.vw[3 * id[v] + c];
                s += ub[r] * rv;
            }
            g[v] = s;
        }
        int na = 0, act[3];
        for (int v = 0; v < 3; ++v)
            if (beta[v] > 1e-12) act[na++] = v;
        if (na == 2) {
            const int iu = act[0], iv = act[1];
            double e[3], pu[3];
            double dd = 0.0, nn = 0.0;
            for (int r = 0; r < 3; ++r) {
                e[r] = X[iv][r] - X[iu][r];
                pu[r] = P[r] - X[iu][r];
                dd += e[r] * e[r];
                nn += pu[r] * e[r];
            }
            const double gt = g[iv] - g[iu];
            for (int r = 0; r < 3; ++r) {
                acc[iu][r] += gt * ((-(e[r] + pu[r]) * dd + 2.0 * nn * e[r]) / (dd * dd));
                acc[iv][r] += gt * ((pu[r] * dd - 2.0 * nn * e[r]) / (dd * dd));
            }
        } else if (na == 3) {
            const double* e0 = V[1];
            const double* e1 = V[2];
            const double* dv = Pr;
            const double s_ = beta[1], t_ = beta[2];
            double m00 = 0, m01 = 0, m11 = 0;
            for (int r = 0; r < 3; ++r) {
                m00 += e0[r] * e0[r];
                m01 += e0[r] * e1[r];
                m11 += e1[r] * e1[r];
            }
            const double g0 = g[1] - g[0], g1 = g[2] - g[0];
            const double det = m00 * m11 - m01 * m01;
            const double z0 = (m11 * g0 - m01 * g1) / det, z1 = (m00 * g1 - m01 * g0) / det;
            for (int r = 0; r < 3; ++r) {
                const double cdd = z0 * e0[r] + z1 * e1[r];
                const double ce0 = z0 * dv[r] - (z0 * (2.0 * s_ * e0[r] + t_ * e1[r]) + z1 * (s_ * e1[r]));
                const double ce1 = z1 * dv[r] - (z0 * (t_ * e0[r]) + z1 * (s_ * e0[r] + 2.0 * t_ * e1[r]));
                acc[0][r] += -cdd - ce0 - ce1;
                acc[1][r] += ce0;
                acc[2][r] += ce1;
            }
        }
    }
    for (int v = 0; v < 3; ++v)
        for (int r = 0; r < 3; ++r)
            if (acc[v][r] != 0.0) atomicAdd(&gX[3 * id[v] + r], acc[v][r]);
}

template <typename T>
__global__ void k_mask_vjp_list(MaskWs m, MaskArgs a, int par, const T* __restrict__ gchi,
                                const T* __restrict__ gus, const T* __restrict__ chi, double* __restrict__ gX) {
    const unsigned long long cnt = m.cnt[par];
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t p = m.list[par][i];
        const int t = m.win[p];
        if (t >= 0 && t < a.n_tri) vjp_point<T>(m, a, p, t, gchi, gus, chi, gX);
    }
}

// dense (tanh) profile: the closest triangle is recomputed per point
template <typename T>
__global__ void k_mask_vjp_dense(MaskWs m, MaskArgs a, const T* __restrict__ gchi, const T* __restrict__ gus,
                                 const T* __restrict__ chi, double* __restrict__ gX) {
    const size_t n = a.n, nz = a.nz, n3 = n * n * nz;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n3; p += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(p % nz), j = (int)((p / nz) % n), i = (int)(p / (n * nz));
        T best = (T)3.0e38;
        int bt = -1;
        for (int t = 0; t < a.n_tri; ++t) {
            const int ia = a.tri[3 * t], ib = a.tri[3 * t + 1], ic = a.tri[3 * t + 2];
            if (ia < 0 || ib < 0 || ic < 0 || ia >= a.n_nodes || ib >= a.n_nodes || ic >= a.n_nodes) continue;
            const double ax = m.xg[3 * ia], ay = m.xg[3 * ia + 1], az = m.xg[3 * ia + 2];
            T P[3] = {(T)(i * a.dx - ax), (T)(j * a.dx - ay), (T)(k * a.dx - az)};
            T A0[3] = {(T)0, (T)0, (T)0};
            T B0[3] = {(T)(m.xg[3 * ib] - ax), (T)(m.xg[3 * ib + 1] - ay), (T)(m.xg[3 * ib + 2] - az)};
            T C0[3] = {(T)(m.xg[3 * ic] - ax), (T)(m.xg[3 * ic + 1] - ay), (T)(m.xg[3 * ic + 2] - az)};
            T bary[3];
            const T d = sqrt(closest_tri<T>(P, A0, B0, C0, bary));
            if (d < best) { best = d; bt = t; }
        }
        if (bt >= 0) vjp_point<T>(m, a, (uint32_t)p, bt, gchi, gus, chi, gX);
    }
}

// grad_xw[v] += R^T gX[v]  (global -> wing frame)
__global__ void k_vjp_to_wing(MaskArgs a, const double* __restrict__ gX, double* __restrict__ gxw) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.n_nodes) return;
    for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        for (int r = 0; r < 3; ++r) s += a.R[3 * r + c] * gX[3 * v + r];
        gxw[3 * v + c] += s;
    }
}

}  // namespace ps
