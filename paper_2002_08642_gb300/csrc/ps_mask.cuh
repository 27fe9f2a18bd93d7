// ps_mask.cuh -- GPU rasteriser of the wing mask chi and the solid velocity
// u_s from the mass-spring wing's triangle mesh (Sec. 4.1):
//   * delta(x) = min over triangles of the distance from grid point x to the
//     triangle, each triangle tested only against the grid points of its
//     bounding box dilated by t_w + h (the mask's reach; no periodic images);
//   * chi(delta) by Eq. (mask_function) (or the tanh profile, evaluated at
//     every point against every triangle);
//   * u_s = V_O + R (sum_v beta_v v_v^(w)) + Omega x (x - X_O) with beta the
//     barycentric coordinates of the closest point on the closest triangle
//     (Eq. relative_velocities).
//
// Banded (cosine) profile, per call:
//   clear     zero chi/u_s and reset the per-point keys of the points the
//             previous call touched (list kept in the workspace), clear the
//             line flags, and the global node positions X_O + R x^(w)
//             (double);
//   tris      per triangle (one thread each): grid-index bounding box and
//             the geometry the pair tests need, in the context precision:
//             vertex a as grid cell + offset, edges b - a and c - a;
//   prefix    exclusive prefix sum of the box point counts (one block);
//   scatter1  for every (triangle, box point) pair with distance < reach:
//             atomicMin of a 64-bit key (non-negative IEEE values order like
//             their bit patterns); the first writer appends the point to the
//             touched list. FP32: the key is the distance bits above the
//             triangle index, so its minimum also names the winner (exact
//             ties -> smallest index). FP64: the distance bits alone, and
//   scatter2  (FP64 only) pairs within a few ulps of the minimum: atomicMin
//             of the triangle index (near-ties -> smallest index);
//   evaluate  per touched point: distance and barycentrics recomputed in
//             double on the winning triangle, chi, u_s, line flags.
// The distance used to pick the winner is computed in the context precision.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace ps {

struct MaskArgs {
    int n, nz;   // grid n x n x nz, spacing dx on every axis
    int x_lo, x_hi;   // x-planes [x_lo, x_hi) rasterised (a slab of the sharded step; 0, n otherwise)
    double dx, tw, h;
    int profile;
    const double* xw;
    const double* vw;
    int n_nodes;
    const int32_t* tri;
    int n_tri;
    double R[9], XO[3], VO[3], Om[3];
};

static constexpr int kMaskMaxTri = 1 << 17;
static constexpr int kMaskMaxNodes = 1 << 17;

// Per-triangle geometry of the pair tests: vertex a = ca dx + f per axis (ca
// its grid cell index, f in [0, dx) the rest), edges b - a and c - a; the
// lengths rounded once from double to T. A grid point minus a is then
// (i - ca) dx - f, with no double arithmetic per pair.
template <typename T> struct TriGeo {
    int ca[4];
    T f[3], b[3], c[3];
};
static constexpr size_t kTriGeoBytes = 128;   // >= sizeof(TriGeo<double>)

// Workspace: keys (8 B/pt), winner ids (4 B/pt), two touched lists (4 B/pt
// each), counters, node and triangle scratch.
inline size_t mask_workspace_bytes(int n, int nz) {
    const size_t n3 = (size_t)n * n * nz;
    auto a = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return a(n3 * 8) + a(n3 * 4) + 2 * a(n3 * 4) + a(64) + a((size_t)kMaskMaxNodes * 3 * 8) +
           a((size_t)kMaskMaxTri * 8 * 4) + a(((size_t)kMaskMaxTri + 1) * 8) + a((size_t)kMaskMaxTri * kTriGeoBytes);
}

struct MaskWs {
    unsigned long long* key;
    int32_t* win;
    uint32_t* list[2];
    unsigned long long* cnt;  // [0],[1]: list lengths, [2]: total pairs, [4]: bad-index flag
    double* xg;
    int32_t* box;              // per triangle: i0,j0,k0,ei,ej,ek, point count (+1 pad)
    unsigned long long* pre;   // exclusive prefix of box sizes (n_tri + 1)
    unsigned char* geo;        // per triangle: TriGeo<T> in kTriGeoBytes
};

inline MaskWs mask_ws_split(unsigned char* w, int n, int nz) {
    const size_t n3 = (size_t)n * n * nz;
    auto a = [](size_t x) { return (x + 255) & ~(size_t)255; };
    MaskWs m;
    size_t o = 0;
    m.key = (unsigned long long*)(w + o); o += a(n3 * 8);
    m.win = (int32_t*)(w + o); o += a(n3 * 4);
    m.list[0] = (uint32_t*)(w + o); o += a(n3 * 4);
    m.list[1] = (uint32_t*)(w + o); o += a(n3 * 4);
    m.cnt = (unsigned long long*)(w + o); o += a(64);
    m.xg = (double*)(w + o); o += a((size_t)kMaskMaxNodes * 3 * 8);
    m.box = (int32_t*)(w + o); o += a((size_t)kMaskMaxTri * 8 * 4);
    m.pre = (unsigned long long*)(w + o); o += a(((size_t)kMaskMaxTri + 1) * 8);
    m.geo = w + o;
    return m;
}

// Closest point of triangle (a, b, c) to p by Voronoi-region tests on the
// vertices, edges and face (the published closest-point-on-triangle method
// of Ericson, Real-Time Collision Detection, Sec. 5.1.5); returns squared
// distance and barycentrics.
template <typename R>
__device__ __forceinline__ R closest_tri(const R p[3], const R a[3], const R b[3], const R c[3], R bary[3]) {
    R ab[3], ac[3], ap[3], bp[3], cp[3];
    for (int i = 0; i < 3; ++i) {
        ab[i] = b[i] - a[i];
        ac[i] = c[i] - a[i];
        ap[i] = p[i] - a[i];
        bp[i] = p[i] - b[i];
        cp[i] = p[i] - c[i];
    }
    auto dot = [](const R* u, const R* v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; };
    const R d1 = dot(ab, ap), d2 = dot(ac, ap);
    R v, w;
    if (d1 <= (R)0 && d2 <= (R)0) { v = 0; w = 0; }
    else {
        const R d3 = dot(ab, bp), d4 = dot(ac, bp);
        const R d5 = dot(ab, cp), d6 = dot(ac, cp);
        const R vc = d1 * d4 - d3 * d2;
        const R vb = d5 * d2 - d1 * d6;
        const R va = d3 * d6 - d5 * d4;
        if (d3 >= (R)0 && d4 <= d3) { v = 1; w = 0; }
        else if (vc <= (R)0 && d1 >= (R)0 && d3 <= (R)0) { v = d1 / (d1 - d3); w = 0; }
        else if (d6 >= (R)0 && d5 <= d6) { v = 0; w = 1; }
        else if (vb <= (R)0 && d2 >= (R)0 && d6 <= (R)0) { v = 0; w = d2 / (d2 - d6); }
        else if (va <= (R)0 && (d4 - d3) >= (R)0 && (d5 - d6) >= (R)0) {
            w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
            v = (R)1 - w;
        } else {
            const R den = (R)1 / (va + vb + vc);
            v = vb * den;
            w = vc * den;
        }
    }
    bary[0] = (R)1 - v - w;
    bary[1] = v;
    bary[2] = w;
    R d2s = 0;
    for (int i = 0; i < 3; ++i) {
        const R q = ap[i] - v * ab[i] - w * ac[i];
        d2s += q * q;
    }
    return d2s;
}

template <typename T> struct KeyBits;
template <> struct KeyBits<float> {
    static __device__ __forceinline__ unsigned long long of(float d) { return (unsigned long long)__float_as_uint(d); }
    static __device__ __forceinline__ float val(unsigned long long k) { return __uint_as_float((unsigned)k); }
};
template <> struct KeyBits<double> {
    static __device__ __forceinline__ unsigned long long of(double d) { return (unsigned long long)__double_as_longlong(d); }
    static __device__ __forceinline__ double val(unsigned long long k) { return __longlong_as_double((long long)k); }
};

// First kernel of a call: zero chi/u_s and reset the key and winner of the
// points the previous call touched (list `par`), clear the line flags
// (n^2 bytes, 16-byte aligned), reset the other list's count, and the
// global node positions X_O + R x^(w) (double).
template <typename T>
__global__ void k_mask_clear(MaskWs m, MaskArgs a, int par, T* chi, T* us, uint8_t* flag, size_t n3, size_t nflag) {
    const unsigned long long tid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long nth = (unsigned long long)gridDim.x * blockDim.x;
    if (tid == 0) m.cnt[par ^ 1] = 0;
    if (tid < (unsigned long long)a.n_nodes) {
        const int i = (int)tid;
        for (int r = 0; r < 3; ++r) {
            double s = a.XO[r];
            for (int c = 0; c < 3; ++c) s += a.R[3 * r + c] * a.xw[3 * i + c];
            m.xg[3 * i + r] = s;
        }
    }
    uint4* f4 = reinterpret_cast<uint4*>(flag);
    for (unsigned long long i = tid; i < nflag / 16; i += nth) f4[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid < nflag % 16) flag[nflag / 16 * 16 + tid] = 0;
    const unsigned long long cnt = m.cnt[par];
    const uint32_t* L = m.list[par];
    for (unsigned long long i = tid; i < cnt; i += nth) {
        const uint32_t p = L[i];
        m.key[p] = ~0ull;
        m.win[p] = 0x7fffffff;
        chi[p] = (T)0;
        for (int c = 0; c < 3; ++c) us[c * n3 + p] = (T)0;
    }
}

// One thread per triangle: bounding box dilated by the reach, its point
// count, and the pair-test geometry.
template <typename T>
__global__ void k_mask_tris(MaskWs m, MaskArgs a, double reach) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_tri) return;
    int ok = 1;
    int id[3];
    double lo[3], hi[3];
    for (int r = 0; r < 3; ++r) { lo[r] = 1e300; hi[r] = -1e300; }
    for (int v = 0; v < 3; ++v) {
        id[v] = a.tri[3 * t + v];
        if (id[v] < 0 || id[v] >= a.n_nodes) { ok = 0; break; }
        for (int r = 0; r < 3; ++r) {
            const double q = m.xg[3 * id[v] + r];
            lo[r] = fmin(lo[r], q);
            hi[r] = fmax(hi[r], q);
        }
    }
    int e[3] = {0, 0, 0}, i0[3] = {0, 0, 0};
    TriGeo<T> gt;
    for (int r = 0; r < 3; ++r) { gt.ca[r] = 0; gt.f[r] = gt.b[r] = gt.c[r] = (T)0; }
    gt.ca[3] = 0;
    if (ok) {
        for (int r = 0; r < 3; ++r) {
            double l = ceil((lo[r] - reach) / a.dx), h = floor((hi[r] + reach) / a.dx);
            l = fmax(l, r == 0 ? (double)a.x_lo : 0.0);
            h = fmin(h, r == 0 ? (double)(a.x_hi - 1) : (double)((r == 2 ? a.nz : a.n) - 1));
            i0[r] = (int)l;
            e[r] = h >= l ? (int)(h - l) + 1 : 0;
            const double ar = m.xg[3 * id[0] + r];
            const double cr = floor(ar / a.dx);
            gt.ca[r] = (int)cr;
            gt.f[r] = (T)(ar - cr * a.dx);
            gt.b[r] = (T)(m.xg[3 * id[1] + r] - ar);
            gt.c[r] = (T)(m.xg[3 * id[2] + r] - ar);
        }
    } else {
        m.cnt[4] = 1;
    }
    int* b = m.box + 8 * t;
    b[0] = i0[0]; b[1] = i0[1]; b[2] = i0[2];
    b[3] = e[0]; b[4] = e[1]; b[5] = e[2];
    b[6] = e[0] * e[1] * e[2];
    *reinterpret_cast<TriGeo<T>*>(m.geo + (size_t)t * kTriGeoBytes) = gt;
}

// One block of 1024 threads: exclusive prefix sum of the box point counts
// (per-thread chunks, then a scan of the chunk totals by warp shuffles).
__global__ void k_mask_prefix(MaskWs m, MaskArgs a) {
    __shared__ unsigned long long wsum[32];
    const int nt = a.n_tri;
    const int per = (nt + blockDim.x - 1) / blockDim.x;
    const int t0 = threadIdx.x * per, t1 = min(nt, t0 + per);
    unsigned long long local = 0;
    for (int t = t0; t < t1; ++t) local += (unsigned long long)m.box[8 * t + 6];
    // inclusive scan within the warp, then of the warp totals
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long inc = local;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        unsigned long long w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += v;
        }
        wsum[lane] = w;   // inclusive totals of warps 0..lane
    }
    __syncthreads();
    unsigned long long run = inc - local + (wid > 0 ? wsum[wid - 1] : 0ull);
    if (threadIdx.x == blockDim.x - 1) {
        m.cnt[2] = run + local;
        m.pre[nt] = run + local;
    }
    for (int t = t0; t < t1; ++t) {
        m.pre[t] = run;
        run += (unsigned long long)m.box[8 * t + 6];
    }
}

__device__ __forceinline__ int find_tri(const unsigned long long* pre, int nt, unsigned long long w) {
    int lo = 0, hi = nt;  // pre[lo] <= w < pre[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= w) lo = mid; else hi = mid;
    }
    return lo;
}

template <typename T>
__device__ __forceinline__ bool pair_dist(const MaskWs& m, const MaskArgs& a, int t, unsigned long long local,
                                          uint32_t* pt, T* dist) {
    const int* b = m.box + 8 * t;
    const uint32_t l = (uint32_t)local, ek = (uint32_t)b[5], ej = (uint32_t)b[4];
    const uint32_t q = l / ek;
    const int k = b[2] + (int)(l - q * ek);
    const int j = b[1] + (int)(q % ej);
    const int i = b[0] + (int)(q / ej);
    const TriGeo<T>& g = *reinterpret_cast<const TriGeo<T>*>(m.geo + (size_t)t * kTriGeoBytes);
    // grid point minus vertex a, from whole cells and the vertex offset
    const T dx = (T)a.dx;
    T P[3] = {(T)(i - g.ca[0]) * dx - g.f[0], (T)(j - g.ca[1]) * dx - g.f[1], (T)(k - g.ca[2]) * dx - g.f[2]};
    T A0[3] = {(T)0, (T)0, (T)0};
    T B0[3] = {g.b[0], g.b[1], g.b[2]};
    T C0[3] = {g.c[0], g.c[1], g.c[2]};
    T bary[3];
    const T d = sqrt(closest_tri<T>(P, A0, B0, C0, bary));
    *pt = (uint32_t)(((size_t)i * a.n + j) * a.nz + k);
    *dist = d;
    return d < (T)(a.tw + a.h);
}

template <typename T>
__global__ void k_mask_scatter1(MaskWs m, MaskArgs a, int par) {
    const unsigned long long W = m.cnt[2];
    for (unsigned long long w = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; w < W;
         w += (unsigned long long)gridDim.x * blockDim.x) {
        const int t = find_tri(m.pre, a.n_tri, w);
        uint32_t p;
        T d;
        if (!pair_dist<T>(m, a, t, w - m.pre[t], &p, &d)) continue;
        // FP32: distance bits above the triangle index, so the minimum key
        // also holds the winner (exact ties -> smallest index); FP64: the
        // distance alone, the winner by k_mask_scatter2
        unsigned long long key = KeyBits<T>::of(d);
        if constexpr (sizeof(T) == 4) key = (key << 32) | (unsigned long long)(uint32_t)t;
        const unsigned long long old = atomicMin(&m.key[p], key);
        if (old == ~0ull) {
            const unsigned long long slot = atomicAdd(&m.cnt[par], 1ull);
            m.list[par][slot] = p;
        }
    }
}

// Pairs within a few units in the last place of the minimum (the same
// distance recomputed here may round differently from the first pass):
// smallest triangle index wins, so near-exact ties go to the smaller index.
template <typename T> struct Ulps;
template <> struct Ulps<float> {
    static __device__ __forceinline__ float of(float d) { return d * 4.8e-7f + 1e-30f; }
};
template <> struct Ulps<double> {
    static __device__ __forceinline__ double of(double d) { return d * 9.0e-16 + 1e-300; }
};

template <typename T>
__global__ void k_mask_scatter2(MaskWs m, MaskArgs a) {
    const unsigned long long W = m.cnt[2];
    for (unsigned long long w = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; w < W;
         w += (unsigned long long)gridDim.x * blockDim.x) {
        const int t = find_tri(m.pre, a.n_tri, w);
        uint32_t p;
        T d;
        if (!pair_dist<T>(m, a, t, w - m.pre[t], &p, &d)) continue;
        const T dmin = KeyBits<T>::val(m.key[p]);
        if (d <= dmin + Ulps<T>::of(dmin)) atomicMin(&m.win[p], t);
    }
}

__device__ __forceinline__ double chi_profile(double d, double tw, double h, int profile) {
    if (profile == 1) return 0.5 * (1.0 - tanh((d - tw) / h));
    if (d <= tw - h) return 1.0;
    if (d >= tw + h) return 0.0;
    return 0.5 * (1.0 + cos(M_PI * (d - tw + h) / (2.0 * h)));
}

// chi and u_s at grid point p from triangle t (double throughout).
template <typename T>
__device__ __forceinline__ void eval_point(const MaskWs& m, const MaskArgs& a, uint32_t p, int t, T* chi, T* us,
                                           uint8_t* flag) {
    const size_t n = a.n, nz = a.nz, n3 = n * n * nz;
    const int k = (int)(p % nz), j = (int)((p / nz) % n), i = (int)(p / (n * nz));
    const double X[3] = {i * a.dx, j * a.dx, k * a.dx};
    const int id[3] = {a.tri[3 * t], a.tri[3 * t + 1], a.tri[3 * t + 2]};
    double P[3], V[3][3];
    for (int v = 0; v < 3; ++v)
        for (int r = 0; r < 3; ++r) V[v][r] = m.xg[3 * id[v] + r] - m.xg[3 * id[0] + r];
    for (int r = 0; r < 3; ++r) P[r] = X[r] - m.xg[3 * id[0] + r];
    double bary[3];
    const double d = sqrt(closest_tri<double>(P, V[0], V[1], V[2], bary));
    const double c = chi_profile(d, a.tw, a.h, a.profile);
    chi[p] = (T)c;
    if (c > 0.0 || a.profile == 1) {
        double vl[3] = {0, 0, 0};
        for (int v = 0; v < 3; ++v)
            for (int r = 0; r < 3; ++r) vl[r] += bary[v] * a.vw[3 * id[v] + r];
        double rr[3];
        for (int r = 0; r < 3; ++r) rr[r] = X[r] - a.XO[r];
        const double rot[3] = {a.Om[1] * rr[2] - a.Om[2] * rr[1], a.Om[2] * rr[0] - a.Om[0] * rr[2],
                               a.Om[0] * rr[1] - a.Om[1] * rr[0]};
        for (int r = 0; r < 3; ++r) {
            double g = a.VO[r] + rot[r];
            for (int cc = 0; cc < 3; ++cc) g += a.R[3 * r + cc] * vl[cc];
            us[r * n3 + p] = (T)g;
        }
        if (c > 0.0) flag[(size_t)i * n + j] = 1;
    }
}

template <typename T>
__global__ void k_mask_eval(MaskWs m, MaskArgs a, int par, T* chi, T* us, uint8_t* flag) {
    const unsigned long long cnt = m.cnt[par];
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t p = m.list[par][i];
        int t;
        if constexpr (sizeof(T) == 4) {   // the winner is the key's low word; kept for the VJP
            t = (int)(uint32_t)m.key[p];
            m.win[p] = t;
        } else {
            t = m.win[p];
        }
        if (t >= 0 && t < a.n_tri) eval_point<T>(m, a, p, t, chi, us, flag);
    }
}

// Dense (tanh) profile: every point against every triangle in index order.
template <typename T>
__global__ void k_mask_dense(MaskWs m, MaskArgs a, T* chi, T* us, uint8_t* flag) {
    const size_t n = a.n, nz = a.nz, n3 = n * n * nz;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n3; p += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(p % nz), j = (int)((p / nz) % n), i = (int)(p / (n * nz));
        if (i < a.x_lo || i >= a.x_hi) continue;
        T best = (T)3.0e38;
        int bt = 0;
        for (int t = 0; t < a.n_tri; ++t) {
            const int ia = a.tri[3 * t], ib = a.tri[3 * t + 1], ic = a.tri[3 * t + 2];
            if (ia < 0 || ib < 0 || ic < 0 || ia >= a.n_nodes || ib >= a.n_nodes || ic >= a.n_nodes) {
                if (p == 0) m.cnt[4] = 1;
                continue;
            }
            const double ax = m.xg[3 * ia], ay = m.xg[3 * ia + 1], az = m.xg[3 * ia + 2];
            T P[3] = {(T)(i * a.dx - ax), (T)(j * a.dx - ay), (T)(k * a.dx - az)};
            T A0[3] = {(T)0, (T)0, (T)0};
            T B0[3] = {(T)(m.xg[3 * ib] - ax), (T)(m.xg[3 * ib + 1] - ay), (T)(m.xg[3 * ib + 2] - az)};
            T C0[3] = {(T)(m.xg[3 * ic] - ax), (T)(m.xg[3 * ic + 1] - ay), (T)(m.xg[3 * ic + 2] - az)};
            T bary[3];
            const T d = sqrt(closest_tri<T>(P, A0, B0, C0, bary));
            if (d < best) { best = d; bt = t; }
        }
        eval_point<T>(m, a, (uint32_t)p, bt, chi, us, flag);
    }
}

// Host driver (in ps_api.cu). `par` is the index of the touched list the
// previous call filled; the call clears those points, fills the other list
// and returns its index in *par_out. `init` resets every key (first call);
// `dense_dirty` zeroes chi/u_s everywhere first (after a dense mask).
template <typename T>
cudaError_t rasterise(const MaskArgs& a, void* chi, void* us, uint8_t* flag, unsigned char* ws, int par, bool init,
                      bool dense_dirty, cudaStream_t s, int* par_out);

}  // namespace ps
