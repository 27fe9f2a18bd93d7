// ps_api.cu -- the C ABI of libps (declared in include/ps.h): context and
// workspace layout, host-side tables, argument checks, dispatch to the
// per-size engines, and the precision-generic reductions (forces, moments,
// diagnostics, mask line flags).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "ps_fault.h"
#include "ps.h"
#include "ps_engine.cuh"
#include "ps_mask.cuh"
#include "ps_adjoint.cuh"
#include "ps_loads.cuh"

using namespace ps;

struct ps_ctx {
    ps_params p;
    cudaStream_t stream;
    int device;
    int fp64;
    const Ops* ops;
    int zblocks;        // force partials written by the z pass
    KP kp;
    Bufs b;
    size_t elem;        // bytes of one real
    size_t ustate;      // bytes of one spectral state array (3 fields)
    double* out;        // device scratch for final reductions (64 doubles)
    unsigned char* mask_ws;   // rasteriser scratch
    size_t mask_ws_bytes;
    int mask_par;             // touched list filled by the last rasterisation
    bool mask_init;           // rasteriser keys initialised
    bool mask_dense_dirty;    // chi/u_s may be nonzero outside the touched list
    CUtensorMap tmA, tmB;     // TMA descriptors of the y passes' inputs
    CUtensorMap tmU, tmA5;    // TMA descriptors of the x passes' inputs
    CUtensorMap tmG;          // adjoint G (x-inverse input), with_adjoint only
    CUtensorMap tmUp, tmHp;   // U and H in x-forward boxes (L2 prefetch)
    CUtensorMap tmN;          // keep_uw: the pressure's N fields (y-forward input)
    bool uw_valid;            // keep_uw: B holds u and omega of the current state
    // adjoint (with_adjoint): lam, mu, G, W, Ub, Wb spectral; u, w, nb physical
    void* adj_spec[6];
    void* adj_phys[3];
    double* gX;               // rasteriser VJP scratch (n_nodes x 3)
    MaskArgs last_mask;       // geometry of the last rasterisation
    bool has_last_mask;
    int nstep;
    int has_velocity;
    // slab of the sharded step (ps_slab_set): x-planes and kept ky rows
    bool slab;
    int slab_x0, slab_x1, slab_ky0, slab_ky1;
    // per-pass timing: a ring of events, kTimingRing steps deep
    bool timing;
    std::vector<cudaEvent_t> tev_step;   // kTimingRing x kEvPerStep
    std::vector<cudaEvent_t> tev_mask;   // kTimingRing x 2
    long t_steps, t_masks;
    std::string err;
};

static const int kTimingRing = 256;
static const char* kPassNames[] = {"x_inverse_curl", "y_inverse", "z_c2r_nonlinear_r2c", "y_forward",
                                   "x_forward_project_ab2", "rasterise"};

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int tile_width(int fp64) { return fp64 ? 8 : 16; }

struct Layout {
    size_t U, H, A, B, N3, chi, us, flag, tw, Ex, Ez, partial, out, err, mask, adj_spec[6], adj_phys[3], gX, total;
    size_t ustate, mask_bytes;
};

int mmax_of(int n) { return (n - 1) / 3; }
// points along z (0 means n)
int nz_of(const ps_params* p) { return p->nz == 0 ? p->n : p->nz; }

bool layout_for(const ps_params* p, const Ops* ops, Layout* L) {
    const int n = p->n, nz = nz_of(p);
    const int fp64 = p->precision == PS_FP64;
    const size_t er = fp64 ? 8 : 4, ec = 2 * er;
    const int mm = mmax_of(n), K = 2 * mm + 1, Kz = mmax_of(nz) + 1;
    const int Cw = tile_width(fp64);
    const int Kzp = (Kz + Cw - 1) / Cw * Cw;
    const size_t n3 = (size_t)n * n * nz;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    L->ustate = 3 * (size_t)K * K * Kzp * ec;
    L->U = take(L->ustate);
    L->H = take(L->ustate);
    L->A = take(6 * (size_t)n * K * Kzp * ec);
    L->B = take(6 * (size_t)n * n * Kzp * ec);
    L->N3 = p->keep_uw ? take(3 * (size_t)n * n * Kzp * ec) : 0;
    L->chi = take(n3 * er);
    L->us = take(3 * n3 * er);
    L->flag = take((size_t)n * n);
    // n-line table, then (n = 3M) the M-line table at n and e^{2 pi i b q/n}
    // at 2n; for nz != n the same three for nz-lines from 3n on
    L->tw = take((size_t)3 * (n + nz) * ec);
    L->Ex = take((size_t)K * er);
    L->Ez = take((size_t)Kz * er);
    const size_t nparts = (size_t)n * n + 4096;
    L->partial = take(nparts * 6 * sizeof(double));
    L->out = take(64 * sizeof(double));
    L->err = take(256);
    L->mask_bytes = mask_workspace_bytes(n, nz);
    L->mask = take(L->mask_bytes);
    // lam, mu, G, (unused), Ub, Wb
    for (int i = 0; i < 6; ++i) L->adj_spec[i] = p->with_adjoint && i != 3 ? take(L->ustate) : 0;
    for (int i = 0; i < 3; ++i) L->adj_phys[i] = p->with_adjoint ? take(3 * n3 * er) : 0;
    L->gX = take((size_t)kMaskMaxNodes * 3 * sizeof(double));
    L->total = off;
    return true;
}

const Ops* ops_for(const ps_params* p) {
    const int nz = nz_of(p);
    const Ops* o = p->precision == PS_FP64 ? ops_f64_a(p->n, nz) : ops_f32_a(p->n, nz);
    if (!o) o = p->precision == PS_FP64 ? ops_f64_b(p->n, nz) : ops_f32_b(p->n, nz);
    return o;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2-D map over `rows` rows of 2 Kzp reals (complex rows of Kzp), box of
// `bc` complex columns by `br` rows.
bool encode_rows(CUtensorMap* tm, void* base, int fp64, size_t rows, int Kzp, int bc, int br) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const size_t er = fp64 ? 8 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)(2 * Kzp), (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(2 * Kzp * er)};
    cuuint32_t box[2] = {(cuuint32_t)(2 * bc), (cuuint32_t)br};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(tm, fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides,
                    box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// 3-D map {2 Kzp reals, d1 rows of stride Kzp complex, d2 planes of stride
// d1 Kzp complex}, box of `bc` complex columns x 1 x `br` planes.
bool encode_planes(CUtensorMap* tm, void* base, int fp64, int Kzp, size_t d1, size_t d2, int bc, int br) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const size_t er = fp64 ? 8 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)(2 * Kzp), (cuuint64_t)d1, (cuuint64_t)d2};
    cuuint64_t strides[2] = {(cuuint64_t)(2 * Kzp * er), (cuuint64_t)(d1 * 2 * Kzp * er)};
    cuuint32_t box[3] = {(cuuint32_t)(2 * bc), 1u, (cuuint32_t)br};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(tm, fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides,
                    box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

ps_status fail(ps_ctx* c, ps_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

ps_status cuda_fail(ps_ctx* c, cudaError_t e, const char* where) {
    return fail(c, PS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

ps_status check_params(const ps_params* p, std::string* why) {
    if (!p) { *why = "null params"; return PS_EINVAL; }
    if (p->precision != PS_FP32 && p->precision != PS_FP64) { *why = "precision must be PS_FP32 or PS_FP64"; return PS_EINVAL; }
    if (p->mask_profile != PS_MASK_COS && p->mask_profile != PS_MASK_TANH) { *why = "bad mask_profile"; return PS_EINVAL; }
    if (p->mean_mode != PS_MEAN_FIXED && p->mean_mode != PS_MEAN_FREE) { *why = "bad mean_mode"; return PS_EINVAL; }
    if (p->with_adjoint != 0 && p->with_adjoint != 1) { *why = "with_adjoint must be 0 or 1"; return PS_EINVAL; }
    if (p->keep_uw != 0 && p->keep_uw != 1) { *why = "keep_uw must be 0 or 1"; return PS_EINVAL; }
    if (!(p->L > 0) || !(p->nu >= 0) || !(p->eta > 0) || !(p->dt > 0) || !(p->h > 0) || !(p->tw >= 0)) {
        *why = "L, eta, dt, h must be > 0 and nu, tw >= 0";
        return PS_EINVAL;
    }
    if (p->nz < 0) { *why = "nz must be >= 0"; return PS_EINVAL; }
    if (!ops_for(p)) {
        *why = "grid size n=" + std::to_string(p->n) + ", nz=" + std::to_string(nz_of(p)) + " is not built into libps";
        return PS_EUNSUPPORTED;
    }
    return PS_OK;
}

// exp(+2 pi i q / n) in double with exact values on the axes.
void unit_root(long q, long n, double* c, double* s) {
    q %= n;
    if (q < 0) q += n;
    // reduce to the first octant via symmetries (q/n in [0, 1/8])
    const long n8 = n, q8 = 8 * q;  // angle = 2 pi q / n; octant = floor(8 q / n)
    long oct = q8 / n8;
    double rem = (double)(q8 - oct * n8) / (double)n8;  // in [0,1): fraction of an octant
    const double qpi4 = 0.78539816339744830962;          // pi / 4
    double a, cb, sb;
    if (oct % 2 == 0) { a = rem * qpi4; cb = cos(a); sb = sin(a); }
    else { a = (1.0 - rem) * qpi4; cb = sin(a); sb = cos(a); }
    // rotate (cb, sb) by oct/2 quarter turns
    switch ((oct / 2) % 4) {
        case 0: *c = cb; *s = sb; break;
        case 1: *c = -sb; *s = cb; break;
        case 2: *c = -cb; *s = -sb; break;
        default: *c = sb; *s = -cb; break;
    }
}

template <typename T>
void host_tables(const ps_params* p, std::vector<unsigned char>& tw, std::vector<unsigned char>& ex,
                 std::vector<unsigned char>& ez) {
    using C2 = cplx<T>;
    const int n = p->n, nz = nz_of(p), mm = mmax_of(n), K = 2 * mm + 1, Kz = mmax_of(nz) + 1;
    std::vector<C2> t((size_t)3 * (n + nz), cmk<C2>((T)0, (T)0));
    // stage twiddles of a length-m line at offset `base`
    auto line_table = [&](int m, size_t base) {
        const int S = n_stages(m);
        for (int s = 1; s < S; ++s) {
            const int r = radix_at(m, s), Ls = ls_at(m, s), o = tw_offset(m, s);
            for (int tt = 1; tt < r; ++tt)
                for (int k = 0; k < Ls; ++k) {
                    double c, sn;
                    unit_root((long)tt * k, (long)Ls * r, &c, &sn);
                    t[base + o + (tt - 1) * Ls + k] = cmk<C2>((T)c, (T)sn);
                }
        }
    };
    // the table of length-m lines at `base`: the stage twiddles, then for
    // m = 3M the M-line table at base + m and e^{2 pi i b q/m} at base + 2m
    auto tables = [&](int m, size_t base) {
        line_table(m, base);
        if (m % 3 == 0) {
            const int M = m / 3;
            line_table(M, base + (size_t)m);
            for (int b = 1; b <= 2; ++b)
                for (int q = 0; q < M; ++q) {
                    double c, sn;
                    unit_root((long)b * q, (long)m, &c, &sn);
                    t[base + (size_t)2 * m + (b - 1) * M + q] = cmk<C2>((T)c, (T)sn);
                }
        }
    };
    tables(n, 0);
    if (nz != n) tables(nz, (size_t)3 * n);
    tw.assign((unsigned char*)t.data(), (unsigned char*)(t.data() + t.size()));
    const double ks = 2.0 * M_PI / p->L;
    const double ksz = ks * (double)n / (double)nz;   // 2 pi / Lz, Lz = L nz / n
    std::vector<T> vx(K), vz(Kz);
    for (int c = 0; c < K; ++c) {
        const int m = c <= mm ? c : c - K;
        vx[c] = (T)exp(-p->nu * (ks * m) * (ks * m) * p->dt);
    }
    for (int c = 0; c < Kz; ++c) vz[c] = (T)exp(-p->nu * (ksz * c) * (ksz * c) * p->dt);
    ex.assign((unsigned char*)vx.data(), (unsigned char*)(vx.data() + K));
    ez.assign((unsigned char*)vz.data(), (unsigned char*)(vz.data() + Kz));
}

// ------------------------------------------------------ generic kernels
template <typename T>
__global__ void k_line_flags(const T* __restrict__ chi, uint8_t* __restrict__ flag, int n, int nz) {
    const long line = (long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (line >= (long)n * n) return;
    int any = 0;
    for (int z = lane; z < nz; z += 32) any |= chi[line * nz + z] != (T)0;
    any = __any_sync(0xffffffffu, any);
    if (lane == 0) flag[line] = (uint8_t)any;
}

// Deterministic final sum of nb x 6 partials (Neumaier), scaled.
__global__ void k_force_final(const double* __restrict__ part, int nb, double scale, double* __restrict__ out) {
    __shared__ double sh[256 * 6];
    Acc a[6] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        for (int i = 0; i < 6; ++i) a[i].add(part[(size_t)b * 6 + i]);
    for (int i = 0; i < 6; ++i) sh[threadIdx.x * 6 + i] = a[i].val();
    __syncthreads();
    if (threadIdx.x < 6) {
        Acc t = {0, 0};
        for (int w = 0; w < (int)blockDim.x; ++w) t.add(sh[w * 6 + threadIdx.x]);
        out[threadIdx.x] = t.val() * scale;
    }
}

// Energy, max |k . c| and a non-finite count over the spectral state.
template <typename T>
__global__ void k_diag(KP kp, const cplx<T>* __restrict__ U, double* __restrict__ part) {
    __shared__ double red[32 * 3];
    const int K = kp.K, Kz = kp.Kz, Kzp = kp.Kzp, mm = kp.mmax;
    const size_t FS = (size_t)K * K * Kzp;
    const size_t tot = (size_t)K * K * Kz;
    Acc e = {0, 0};
    double dmax = 0.0, bad = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
        const int cz = (int)(i % Kz);
        const size_t r = i / Kz;
        const int cy = (int)(r % K), cx = (int)(r / K);
        const size_t o = ((size_t)cy * K + cx) * Kzp + cz;
        const double kx = kp.ks * cmode_of(cx, mm, K), ky = kp.ks * cmode_of(cy, mm, K), kz = kp.ksz * cz;
        double s = 0.0, dr = 0.0, di = 0.0;
        const double kk[3] = {kx, ky, kz};
        for (int f = 0; f < 3; ++f) {
            const cplx<T> v = U[f * FS + o];
            const double vr = (double)v.x, vi = (double)v.y;
            if (!isfinite(vr) || !isfinite(vi)) bad += 1.0;
            s += vr * vr + vi * vi;
            dr += kk[f] * vr;
            di += kk[f] * vi;
        }
        e.add((cz == 0 ? 1.0 : 2.0) * s);
        const double d = sqrt(dr * dr + di * di);
        dmax = d > dmax ? d : dmax;
    }
    double v[3] = {e.val(), 0.0, bad};
    // max over the block
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, o));
    __shared__ double mx[32];
    if ((threadIdx.x & 31) == 0) mx[threadIdx.x >> 5] = dmax;
    block_sum<3>(v, part + (size_t)blockIdx.x * 3, red);
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) m = fmax(m, mx[w]);
        part[(size_t)blockIdx.x * 3 + 1] = m;
    }
}

// Test hook: an mbarrier that expects 16 bytes of bulk copy that no copy
// delivers (none is issued), waited on with the kernels' bounded wait and a
// caller-chosen cap; on giving up the block records the device error flag
// the way the transform passes do. Nothing is in flight when it returns.
__global__ void k_wait_timeout(int* __restrict__ err, uint32_t cap) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16);
    __syncthreads();
    const bool ok = mbar_wait_cap(&bar, 0, cap);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(err, 1);
}

__global__ void k_diag_final(const double* __restrict__ part, int nb, double half_L3, double* __restrict__ out) {
    if (threadIdx.x != 0) return;
    Acc e = {0, 0};
    double m = 0.0, bad = 0.0;
    for (int b = 0; b < nb; ++b) {
        e.add(part[(size_t)b * 3]);
        m = fmax(m, part[(size_t)b * 3 + 1]);
        bad += part[(size_t)b * 3 + 2];
    }
    out[0] = e.val() * half_L3;
    out[1] = m;
    out[2] = bad;
}

ps_status sync(ps_ctx* c, const char* where) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, where);
    return PS_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

// Grid-stride launches of the rasteriser and its VJP are sized as multiples
// of the GB300's 152 SMs (8 or 16 blocks per SM); any grid is correct.
constexpr int kRasterSM = 152;

template <typename T>
cudaError_t ps::rasterise(const MaskArgs& a, void* chi, void* us, uint8_t* flag, unsigned char* ws, int par, bool init,
                          bool dense_dirty, cudaStream_t s, int* par_out) {
    const size_t n = a.n, n3 = n * n * a.nz;
    MaskWs m = mask_ws_split(ws, a.n, a.nz);
    cudaError_t e;
    if (init) {
        if ((e = cudaMemsetAsync(m.key, 0xff, n3 * 8, s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(m.win, 0x7f, n3 * 4, s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(m.cnt, 0, 64, s)) != cudaSuccess) return e;
    }
    if (dense_dirty) {
        if ((e = cudaMemsetAsync(chi, 0, n3 * sizeof(T), s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(us, 0, 3 * n3 * sizeof(T), s)) != cudaSuccess) return e;
    }
    // the previous call's points, the line flags, the other list's count
    // and the node positions
    const int np = par ^ 1;
    const int cb = (a.n_nodes + 255) / 256 > 8 * kRasterSM ? (a.n_nodes + 255) / 256 : 8 * kRasterSM;
    k_mask_clear<T><<<cb, 256, 0, s>>>(m, a, par, (T*)chi, (T*)us, flag, n3, n * n);
    if (a.profile == PS_MASK_TANH) {
        k_mask_dense<T><<<16 * kRasterSM, 128, 0, s>>>(m, a, (T*)chi, (T*)us, flag);
        *par_out = np;  // both lists empty: the next call must clear densely
        return cudaGetLastError();
    }
    k_mask_tris<T><<<a.n_tri > 0 ? (a.n_tri + 127) / 128 : 1, 128, 0, s>>>(m, a, a.tw + a.h);
    k_mask_prefix<<<1, 1024, 0, s>>>(m, a);
    k_mask_scatter1<T><<<16 * kRasterSM, 256, 0, s>>>(m, a, np);
    if constexpr (sizeof(T) == 8) k_mask_scatter2<T><<<16 * kRasterSM, 256, 0, s>>>(m, a);
    k_mask_eval<T><<<8 * kRasterSM, 256, 0, s>>>(m, a, np, (T*)chi, (T*)us, flag);
    *par_out = np;
    return cudaGetLastError();
}

template cudaError_t ps::rasterise<float>(const MaskArgs&, void*, void*, uint8_t*, unsigned char*, int, bool, bool,
                                          cudaStream_t, int*);
template cudaError_t ps::rasterise<double>(const MaskArgs&, void*, void*, uint8_t*, unsigned char*, int, bool, bool,
                                           cudaStream_t, int*);

template <typename T>
static cudaError_t adjoint_step_t(ps_ctx* c, const AdjW& aw, void* gchi, void* gus) {
    using C2 = cplx<T>;
    cudaStream_t s = c->stream;
    // grid-stride passes: exactly the blocks that are resident at once
    static int spec1_blocks = 0, spec2_blocks = 0, pt_blocks = 0;
    if (pt_blocks == 0) {
        int nsm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
        if (nsm < 1) nsm = 1;
        auto resident = [&](auto kern) {
            int occ = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0);
            return (occ > 0 ? occ : 1) * nsm;
        };
        spec1_blocks = resident(k_adj_spec1<T>);
        spec2_blocks = resident(k_adj_spec2<T>);
        pt_blocks = resident(k_adj_point<T>);
    }
    C2* lam = (C2*)c->adj_spec[0];
    C2* mu = (C2*)c->adj_spec[1];
    C2* G = (C2*)c->adj_spec[2];
    C2* Ub = (C2*)c->adj_spec[4];
    C2* Wb = (C2*)c->adj_spec[5];
    T* up = (T*)c->adj_phys[0];
    T* wp = (T*)c->adj_phys[1];
    T* np_ = (T*)c->adj_phys[2];
    cudaError_t e;
    k_adj_spec1<T><<<spec1_blocks, 256, 0, s>>>(c->kp, lam, mu, G, (const T*)c->b.Ex, (const T*)c->b.Ez, aw.first);
    if ((e = c->ops->inv_uw(c->kp, c->b, up, wp, s)) != cudaSuccess) return e;
    if ((e = c->ops->inv_g(c->kp, c->b, np_, s)) != cudaSuccess) return e;
    k_adj_point<T><<<pt_blocks, 256, 0, s>>>(c->kp, aw, up, wp, np_, (const T*)c->b.chi, (const T*)c->b.us, (T*)gchi,
                                          (T*)gus);
    if ((e = c->ops->fwd3(c->kp, c->b, up, Ub, s)) != cudaSuccess) return e;
    if ((e = c->ops->fwd3(c->kp, c->b, wp, Wb, s)) != cudaSuccess) return e;
    k_adj_spec2<T><<<spec2_blocks, 256, 0, s>>>(c->kp, lam, Ub, Wb);
    return cudaGetLastError();
}

extern "C" {

ps_status ps_supported_n(int32_t* out, int32_t cap, int32_t* count) {
    if (!count) return PS_EINVAL;
    int32_t sizes[] = {
#define PS_LIST(n) n,
        PS_SIZES(PS_LIST)
#undef PS_LIST
    };
    const int32_t total = (int32_t)(sizeof(sizes) / sizeof(sizes[0]));
    std::sort(sizes, sizes + total);
    *count = total;
    if (out)
        for (int32_t i = 0; i < total && i < cap; ++i) out[i] = sizes[i];
    return PS_OK;
}

ps_status ps_workspace_size(const ps_params* p, size_t* bytes) {
    std::string why;
    if (!bytes) return PS_EINVAL;
    ps_status st = check_params(p, &why);
    if (st != PS_OK) return st;
    Layout L;
    layout_for(p, ops_for(p), &L);
    *bytes = L.total;
    return PS_OK;
}

ps_status ps_init(const ps_params* p, void* cuda_stream, void* workspace_dev, size_t workspace_bytes,
                  ps_ctx** out) {
    if (!out) return PS_EINVAL;
    *out = nullptr;
    std::string why;
    ps_status st = check_params(p, &why);
    if (st != PS_OK) return st;
    if (!workspace_dev || ((uintptr_t)workspace_dev & 255)) return PS_EINVAL;
    const Ops* ops = ops_for(p);
    Layout L;
    layout_for(p, ops, &L);
    if (workspace_bytes < L.total) return PS_ENOMEM;

    ps_ctx* c = ps_fault_alloc("ctx") ? nullptr : new (std::nothrow) ps_ctx();
    if (!c) return PS_ENOMEM;
    c->p = *p;
    c->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&c->device);
    c->fp64 = p->precision == PS_FP64;
    c->ops = ops;
    c->elem = c->fp64 ? 8 : 4;
    c->ustate = L.ustate;
    const int n = p->n, nz = nz_of(p), mm = mmax_of(n);
    c->p.nz = nz;
    KP& kp = c->kp;
    kp.n = n;
    kp.nz = nz;
    kp.mmax = mm;
    kp.K = 2 * mm + 1;
    kp.Kz = mmax_of(nz) + 1;
    const int Cw = tile_width(c->fp64);
    // the same rounding as Geo<T, nz>::KZP: the kernels size their staging
    // buffers with that compile-time width and stride lines by kp.Kzp
    kp.Kzp = (kp.Kz + Cw - 1) / Cw * Cw;
    kp.ks = 2.0 * M_PI / p->L;
    const double Lz = p->L * (double)nz / (double)n;
    kp.ksz = 2.0 * M_PI / Lz;
    kp.dt = p->dt;
    kp.inv_eta = 1.0 / p->eta;
    kp.invn3 = 1.0 / ((double)n * n * nz);
    kp.dx = p->L / n;
    kp.half_L3 = 0.5 * p->L * p->L * Lz;
    for (int i = 0; i < 3; ++i) kp.x0[i] = p->x0[i];
    kp.mean_free = p->mean_mode == PS_MEAN_FREE;

    unsigned char* w = (unsigned char*)workspace_dev;
    c->b.U = w + L.U;
    c->b.H = w + L.H;
    c->b.A = w + L.A;
    c->b.B = w + L.B;
    c->b.N3 = p->keep_uw ? (void*)(w + L.N3) : nullptr;
    c->b.tmN = nullptr;
    c->uw_valid = false;
    c->b.chi = w + L.chi;
    c->b.us = w + L.us;
    c->b.flag = (uint8_t*)(w + L.flag);
    c->b.tw = w + L.tw;
    c->b.Ex = w + L.Ex;
    c->b.Ez = w + L.Ez;
    c->b.partial = (double*)(w + L.partial);
    c->out = (double*)(w + L.out);
    c->b.err = (int*)(w + L.err);
    c->mask_ws = w + L.mask;
    for (int i = 0; i < 6; ++i) c->adj_spec[i] = p->with_adjoint && i != 3 ? (void*)(w + L.adj_spec[i]) : nullptr;
    for (int i = 0; i < 3; ++i) c->adj_phys[i] = p->with_adjoint ? (void*)(w + L.adj_phys[i]) : nullptr;
    c->gX = (double*)(w + L.gX);
    c->mask_ws_bytes = L.mask_bytes;

    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (nsm < 1) nsm = 1;
    cudaError_t e = ops->prepare(nsm, &c->zblocks);
    kp.part_off = 0;
    kp.xs0 = 0;
    kp.xsn = n;
    kp.ky0 = 0;
    kp.kyn = kp.K;
    if (e == cudaSuccess) {
        const int Kk = 2 * mm + 1;
        if (!encode_planes(&c->tmA, c->b.A, c->fp64, kp.Kzp, (size_t)n, (size_t)6 * Kk, ops->cy2, ops->br2) ||
            !encode_rows(&c->tmB, c->b.B, c->fp64, (size_t)6 * n * n, kp.Kzp, ops->cy4, ops->br4) ||
            !encode_rows(&c->tmU, c->b.U, c->fp64, (size_t)3 * Kk * Kk, kp.Kzp, ops->cx1, ops->br2) ||
            !encode_rows(&c->tmA5, c->b.A, c->fp64, (size_t)6 * Kk * n, kp.Kzp, ops->cx5, ops->br4) ||
            !encode_rows(&c->tmUp, c->b.U, c->fp64, (size_t)3 * Kk * Kk, kp.Kzp, ops->cx5, ops->br2) ||
            !encode_rows(&c->tmHp, c->b.H, c->fp64, (size_t)3 * Kk * Kk, kp.Kzp, ops->cx5, ops->br2)) {
            delete c;
            return PS_ECUDA;
        }
        c->b.tmA = &c->tmA;
        c->b.tmB = &c->tmB;
        c->b.tmU = &c->tmU;
        c->b.tmA5 = &c->tmA5;
        c->b.tmUp = &c->tmUp;
        c->b.tmHp = &c->tmHp;
        c->b.tmG = nullptr;
        c->b.chi_sp = nullptr;
        if (p->with_adjoint) {
            if (!encode_rows(&c->tmG, c->adj_spec[2], c->fp64, (size_t)3 * Kk * Kk, kp.Kzp, ops->cx1, ops->br2)) {
                delete c;
                return PS_ECUDA;
            }
            c->b.tmG = &c->tmG;
        }
        if (p->keep_uw) {
            if (!encode_rows(&c->tmN, c->b.N3, c->fp64, (size_t)3 * n * n, kp.Kzp, ops->cy4, ops->br4)) {
                delete c;
                return PS_ECUDA;
            }
            c->b.tmN = &c->tmN;
        }
    }
    if (e != cudaSuccess) { ps_status s = cuda_fail(c, e, "kernel attributes"); delete c; return s; }
    std::vector<unsigned char> tw, ex, ez;
    if (c->fp64) host_tables<double>(p, tw, ex, ez);
    else host_tables<float>(p, tw, ex, ez);
    if ((e = cudaMemsetAsync(workspace_dev, 0, L.total, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->b.tw, tw.data(), tw.size(), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->b.Ex, ex.data(), ex.size(), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->b.Ez, ez.data(), ez.size(), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess) {
        delete c;
        return PS_ECUDA;
    }
    *out = c;
    return PS_OK;
}

ps_status ps_destroy(ps_ctx* c) {
    if (!c) return PS_EINVAL;
    for (cudaEvent_t ev : c->tev_step) cudaEventDestroy(ev);
    for (cudaEvent_t ev : c->tev_mask) cudaEventDestroy(ev);
    delete c;
    return PS_OK;
}

ps_status ps_set_velocity(ps_ctx* c, const void* u) {
    if (!c) return PS_EINVAL;
    c->uw_valid = false;   // overwrites B (or the state it was taken from)
    if (!u) return fail(c, PS_EINVAL, "ps_set_velocity: null u");
    DeviceGuard dg(c->device);
    cudaError_t e = c->ops->set_velocity(c->kp, c->b, u, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ps_set_velocity");
    c->nstep = 0;
    c->has_velocity = 1;
    return PS_OK;
}

ps_status ps_get_velocity(ps_ctx* c, void* u) {
    if (!c) return PS_EINVAL;
    c->uw_valid = false;   // overwrites B (or the state it was taken from)
    if (!u) return fail(c, PS_EINVAL, "ps_get_velocity: null u");
    DeviceGuard dg(c->device);
    cudaError_t e = c->ops->get_velocity(c->kp, c->b, u, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ps_get_velocity");
    return PS_OK;
}

ps_status ps_set_mask(ps_ctx* c, const void* chi, const void* us) {
    if (!c) return PS_EINVAL;
    if (!chi || !us) return fail(c, PS_EINVAL, "ps_set_mask: null chi or us");
    DeviceGuard dg(c->device);
    const int n = c->p.n;
    const size_t n3 = (size_t)n * n * c->p.nz;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(c->b.chi, chi, n3 * c->elem, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->b.us, us, 3 * n3 * c->elem, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "ps_set_mask copy");
    const long lines = (long)n * n;
    const int per = 8;  // lines per block (one warp each)
    if (c->fp64) k_line_flags<double><<<(unsigned)((lines + per - 1) / per), 32 * per, 0, c->stream>>>((const double*)c->b.chi, c->b.flag, n, c->p.nz);
    else k_line_flags<float><<<(unsigned)((lines + per - 1) / per), 32 * per, 0, c->stream>>>((const float*)c->b.chi, c->b.flag, n, c->p.nz);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "ps_set_mask flags");
    c->mask_dense_dirty = true;
    c->has_last_mask = false;
    return PS_OK;
}

ps_status ps_get_mask(ps_ctx* c, void* chi, void* us) {
    if (!c) return PS_EINVAL;
    if (!chi || !us) return fail(c, PS_EINVAL, "ps_get_mask: null chi or us");
    DeviceGuard dg(c->device);
    const int n = c->p.n;
    const size_t n3 = (size_t)n * n * c->p.nz;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(chi, c->b.chi, n3 * c->elem, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(us, c->b.us, 3 * n3 * c->elem, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "ps_get_mask");
    return PS_OK;
}

ps_status ps_set_mask_from_nodes(ps_ctx* c, const double* xw, const double* vw, int32_t n_nodes,
                                 const int32_t* tri, int32_t n_tri, const ps_frame* frame) {
    if (!c) return PS_EINVAL;
    if (!xw || !vw || !tri || !frame || n_nodes < 3 || n_tri < 1)
        return fail(c, PS_EINVAL, "ps_set_mask_from_nodes: null pointer or empty mesh");
    DeviceGuard dg(c->device);
    MaskArgs a;
    a.n = c->p.n;
    a.nz = c->p.nz;
    a.x_lo = c->slab ? c->slab_x0 : 0;
    a.x_hi = c->slab ? c->slab_x1 : c->p.n;
    a.dx = c->kp.dx;
    a.tw = c->p.tw;
    a.h = c->p.h;
    a.profile = c->p.mask_profile;
    a.xw = xw;
    a.vw = vw;
    a.n_nodes = n_nodes;
    a.tri = tri;
    a.n_tri = n_tri;
    memcpy(a.R, frame->R, sizeof(a.R));
    memcpy(a.XO, frame->X_O, sizeof(a.XO));
    memcpy(a.VO, frame->V_O, sizeof(a.VO));
    memcpy(a.Om, frame->Omega, sizeof(a.Om));
    if (n_tri > kMaskMaxTri || n_nodes > kMaskMaxNodes)
        return fail(c, PS_EINVAL, "ps_set_mask_from_nodes: more than 131072 triangles or nodes");
    int np = 0;
    cudaEvent_t* ev = nullptr;
    if (c->timing) {
        ev = &c->tev_mask[(size_t)(c->t_masks++ % kTimingRing) * 2];
        cudaEventRecord(ev[0], c->stream);
    }
    cudaError_t e = c->fp64 ? rasterise<double>(a, c->b.chi, c->b.us, c->b.flag, c->mask_ws, c->mask_par, !c->mask_init,
                                                c->mask_dense_dirty, c->stream, &np)
                            : rasterise<float>(a, c->b.chi, c->b.us, c->b.flag, c->mask_ws, c->mask_par, !c->mask_init,
                                               c->mask_dense_dirty, c->stream, &np);
    if (e != cudaSuccess) return cuda_fail(c, e, "ps_set_mask_from_nodes");
    if (ev) cudaEventRecord(ev[1], c->stream);
    c->mask_par = np;
    c->mask_init = true;
    c->last_mask = a;
    c->has_last_mask = true;
    c->mask_dense_dirty = (a.profile == PS_MASK_TANH);
    return PS_OK;
}

ps_status ps_step(ps_ctx* c, int32_t nsteps) {
    if (!c) return PS_EINVAL;
    if (nsteps < 0) return fail(c, PS_EINVAL, "ps_step: nsteps < 0");
    if (!c->has_velocity) return fail(c, PS_ESTATE, "ps_step: no velocity set");
    DeviceGuard dg(c->device);
    for (int i = 0; i < nsteps; ++i) {
        cudaEvent_t* ev = nullptr;
        if (c->timing) ev = &c->tev_step[(size_t)(c->t_steps++ % kTimingRing) * kEvPerStep];
        const int resume = c->uw_valid ? 1 : 0;
        c->uw_valid = false;   // the step's z pass overwrites u in B
        cudaError_t e = c->ops->step(c->kp, c->b, c->nstep == 0, resume, c->stream, ev);
        if (e != cudaSuccess) return cuda_fail(c, e, "ps_step");
        c->nstep++;
    }
    return PS_OK;
}

ps_status ps_set_sponge(ps_ctx* c, const void* chi_sp_dev, double c_sp) {
    if (!c) return PS_EINVAL;
    if (!chi_sp_dev) {
        c->b.chi_sp = nullptr;
        return PS_OK;
    }
    if (!(c_sp > 0.0)) return fail(c, PS_EINVAL, "ps_set_sponge: C_sp must be > 0");
    c->b.chi_sp = chi_sp_dev;
    c->kp.inv_csp = 1.0 / c_sp;
    return PS_OK;
}

ps_status ps_pressure(ps_ctx* c, void* p_dev) {
    if (!c) return PS_EINVAL;
    if (!p_dev) return fail(c, PS_EINVAL, "ps_pressure: null output");
    if (!c->has_velocity) return fail(c, PS_ESTATE, "ps_pressure: no velocity set");
    DeviceGuard dg(c->device);
    const int resume = c->uw_valid ? 1 : 0;
    c->uw_valid = false;
    cudaError_t e = c->ops->pressure(c->kp, c->b, p_dev, resume, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ps_pressure");
    c->uw_valid = c->b.N3 != nullptr;   // keep_uw: B still holds u and omega of the state
    return PS_OK;
}

ps_status ps_pressure_loads(ps_ctx* c, const void* p_dev, const double* xw, int32_t n_nodes, const int32_t* tri,
                            int32_t n_tri, const ps_frame* frame, double* p_nodes_dev, double* f_nodes_dev) {
    if (!c) return PS_EINVAL;
    if (!p_dev || !xw || !tri || !frame || !p_nodes_dev || !f_nodes_dev || n_nodes < 1 || n_tri < 1)
        return fail(c, PS_EINVAL, "ps_pressure_loads: null pointer or empty mesh");
    if (n_tri > kMaskMaxTri || n_nodes > kMaskMaxNodes)
        return fail(c, PS_EINVAL, "ps_pressure_loads: more than 131072 triangles or nodes");
    DeviceGuard dg(c->device);
    LoadArgs a;
    a.n = c->p.n;
    a.nz = c->p.nz;
    a.dx = c->kp.dx;
    a.xw = xw;
    a.n_nodes = n_nodes;
    a.tri = tri;
    a.n_tri = n_tri;
    memcpy(a.R, frame->R, sizeof(a.R));
    memcpy(a.XO, frame->X_O, sizeof(a.XO));
    const int nb = (n_nodes + 127) / 128;
    if (c->fp64) k_node_pressure<double><<<nb, 128, 0, c->stream>>>(a, (const double*)p_dev, p_nodes_dev);
    else k_node_pressure<float><<<nb, 128, 0, c->stream>>>(a, (const float*)p_dev, p_nodes_dev);
    k_node_loads<<<(n_nodes + 3) / 4, 128, 0, c->stream>>>(a, p_nodes_dev, f_nodes_dev);   // a warp per node
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "ps_pressure_loads");
    return PS_OK;
}

ps_status ps_forces(ps_ctx* c, double F[3], double M[3]) {
    if (!c) return PS_EINVAL;
    if (!F || !M) return fail(c, PS_EINVAL, "ps_forces: null output");
    if (c->nstep == 0) return fail(c, PS_ESTATE, "ps_forces: no step taken yet");
    DeviceGuard dg(c->device);
    const double dx = c->kp.dx;
    k_force_final<<<1, 256, 0, c->stream>>>(c->b.partial, c->zblocks, dx * dx * dx / c->p.eta, c->out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "ps_forces");
    double h[6];
    int derr = 0;
    if ((e = cudaMemcpyAsync(h, c->out, sizeof(h), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&derr, c->b.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "ps_forces copy");
    ps_status s = sync(c, "ps_forces");
    if (s != PS_OK) return s;
    if (derr) return fail(c, PS_ECUDA, "a device-side copy wait gave up (results of the affected steps are invalid)");
    for (int i = 0; i < 3; ++i) { F[i] = h[i]; M[i] = h[3 + i]; }
    return PS_OK;
}

ps_status ps_grid_info(const ps_ctx* c, int32_t* K, int32_t* Kz, int32_t* Kzp) {
    if (!c || !K || !Kz || !Kzp) return PS_EINVAL;
    *K = c->kp.K;
    *Kz = c->kp.Kz;
    *Kzp = c->kp.Kzp;
    return PS_OK;
}

ps_status ps_slab_set(ps_ctx* c, int32_t x0, int32_t x1, int32_t ky0, int32_t ky1) {
    if (!c) return PS_EINVAL;
    const int n = c->p.n, K = c->kp.K, za = c->ops->zalign;
    if (x0 < 0 || x1 > n || x0 >= x1 || ky0 < 0 || ky1 > K || ky0 >= ky1)
        return fail(c, PS_EINVAL, "ps_slab_set: empty or out-of-range slab");
    if (((long)x0 * n) % za != 0 || ((long)x1 * n) % za != 0)
        return fail(c, PS_EINVAL, "ps_slab_set: x-plane bounds times n must be multiples of " + std::to_string(za));
    c->slab = true;
    c->slab_x0 = x0;
    c->slab_x1 = x1;
    c->slab_ky0 = ky0;
    c->slab_ky1 = ky1;
    c->uw_valid = false;
    return PS_OK;
}

ps_status ps_slab_phase(ps_ctx* c, int32_t phase) {
    if (!c) return PS_EINVAL;
    if (!c->slab) return fail(c, PS_ESTATE, "ps_slab_phase: no slab set (ps_slab_set)");
    if (phase < 0 || phase > 2) return fail(c, PS_EINVAL, "ps_slab_phase: phase must be 0, 1 or 2");
    if (!c->has_velocity) return fail(c, PS_ESTATE, "ps_slab_phase: no velocity set");
    DeviceGuard dg(c->device);
    c->uw_valid = false;
    KP k = c->kp;
    k.xs0 = c->slab_x0;
    k.xsn = c->slab_x1 - c->slab_x0;
    k.ky0 = c->slab_ky0;
    k.kyn = c->slab_ky1 - c->slab_ky0;
    k.part_off = 0;
    cudaError_t e = c->ops->slab_phase(k, c->b, phase, c->nstep == 0, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ps_slab_phase");
    if (phase == 2) c->nstep++;
    return PS_OK;
}

ps_status ps_slab_buffer(ps_ctx* c, void** a_dev, size_t* bytes) {
    if (!c || !a_dev || !bytes) return PS_EINVAL;
    *a_dev = c->b.A;
    *bytes = (size_t)6 * c->kp.K * c->p.n * c->kp.Kzp * 2 * c->elem;
    return PS_OK;
}

ps_status ps_clear_error(ps_ctx* c) {
    if (!c) return PS_EINVAL;
    DeviceGuard dg(c->device);
    cudaError_t e = cudaMemsetAsync(c->b.err, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ps_clear_error");
    c->err.clear();
    return sync(c, "ps_clear_error");
}

ps_status ps_debug_wait_timeout(ps_ctx* c, int32_t cap) {
    if (!c) return PS_EINVAL;
    if (cap < 1) return fail(c, PS_EINVAL, "ps_debug_wait_timeout: cap < 1");
    DeviceGuard dg(c->device);
    k_wait_timeout<<<1, 64, 0, c->stream>>>(c->b.err, (uint32_t)cap);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "ps_debug_wait_timeout");
    return sync(c, "ps_debug_wait_timeout");
}

ps_status ps_diagnostics(ps_ctx* c, double* energy, double* max_div) {
    if (!c) return PS_EINVAL;
    if (!energy || !max_div) return fail(c, PS_EINVAL, "ps_diagnostics: null output");
    DeviceGuard dg(c->device);
    const int nb = 304;
    if (c->fp64) k_diag<double><<<nb, 256, 0, c->stream>>>(c->kp, (const double2*)c->b.U, c->b.partial);
    else k_diag<float><<<nb, 256, 0, c->stream>>>(c->kp, (const float2*)c->b.U, c->b.partial);
    k_diag_final<<<1, 32, 0, c->stream>>>(c->b.partial, nb, c->kp.half_L3, c->out + 8);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "ps_diagnostics");
    double h[3];
    if ((e = cudaMemcpyAsync(h, c->out + 8, sizeof(h), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "ps_diagnostics copy");
    ps_status s = sync(c, "ps_diagnostics");
    if (s != PS_OK) return s;
    *energy = h[0];
    *max_div = h[1];
    if (h[2] != 0.0) return fail(c, PS_ENUMERIC, "ps_diagnostics: state holds NaN or Inf");
    return PS_OK;
}

ps_status ps_state_size(const ps_ctx* c, size_t* bytes) {
    if (!c || !bytes) return PS_EINVAL;
    *bytes = 256 + 2 * c->ustate;
    return PS_OK;
}

ps_status ps_save_state(ps_ctx* c, void* buf) {
    if (!c) return PS_EINVAL;
    if (!buf || ((uintptr_t)buf & 15)) return fail(c, PS_EINVAL, "ps_save_state: null or unaligned buffer");
    DeviceGuard dg(c->device);
    unsigned char* d = (unsigned char*)buf;
    int64_t hdr[2] = {c->nstep, c->has_velocity};
    cudaError_t e;
    if ((e = cudaMemcpyAsync(d, hdr, sizeof(hdr), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d + 256, c->b.U, c->ustate, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d + 256 + c->ustate, c->b.H, c->ustate, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "ps_save_state");
    return sync(c, "ps_save_state");
}

ps_status ps_restore_state(ps_ctx* c, const void* buf) {
    if (!c) return PS_EINVAL;
    c->uw_valid = false;   // overwrites B (or the state it was taken from)
    if (!buf || ((uintptr_t)buf & 15)) return fail(c, PS_EINVAL, "ps_restore_state: null or unaligned buffer");
    DeviceGuard dg(c->device);
    const unsigned char* d = (const unsigned char*)buf;
    int64_t hdr[2];
    cudaError_t e;
    if ((e = cudaMemcpyAsync(hdr, d, sizeof(hdr), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->b.U, d + 256, c->ustate, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->b.H, d + 256 + c->ustate, c->ustate, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "ps_restore_state");
    ps_status s = sync(c, "ps_restore_state");
    if (s != PS_OK) return s;
    c->nstep = (int)hdr[0];
    c->has_velocity = (int)hdr[1];
    return PS_OK;
}

ps_status ps_adjoint_reset(ps_ctx* c) {
    if (!c) return PS_EINVAL;
    c->uw_valid = false;   // overwrites B (or the state it was taken from)
    if (!c->p.with_adjoint) return fail(c, PS_ESTATE, "ps_adjoint_reset: context created without with_adjoint");
    DeviceGuard dg(c->device);
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->adj_spec[0], 0, c->ustate, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->adj_spec[1], 0, c->ustate, c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "ps_adjoint_reset");
    return PS_OK;
}

ps_status ps_adjoint_step(ps_ctx* c, const double dJdF[3], const double dJdM[3], int32_t first, void* grad_chi_dev,
                          void* grad_us_dev) {
    if (!c) return PS_EINVAL;
    c->uw_valid = false;   // overwrites B (or the state it was taken from)
    if (!c->p.with_adjoint) return fail(c, PS_ESTATE, "ps_adjoint_step: context created without with_adjoint");
    if (!dJdF || !dJdM || !grad_chi_dev || !grad_us_dev)
        return fail(c, PS_EINVAL, "ps_adjoint_step: null argument");
    DeviceGuard dg(c->device);
    AdjW aw;
    for (int i = 0; i < 3; ++i) { aw.a[i] = dJdF[i]; aw.b[i] = dJdM[i]; }
    aw.first = first ? 1 : 0;
    cudaError_t e = c->fp64 ? adjoint_step_t<double>(c, aw, grad_chi_dev, grad_us_dev)
                            : adjoint_step_t<float>(c, aw, grad_chi_dev, grad_us_dev);
    if (e != cudaSuccess) return cuda_fail(c, e, "ps_adjoint_step");
    return PS_OK;
}

ps_status ps_mask_nodes_vjp(ps_ctx* c, const void* grad_chi_dev, const void* grad_us_dev, double* grad_xw_dev) {
    if (!c) return PS_EINVAL;
    c->uw_valid = false;   // overwrites B (or the state it was taken from)
    if (!grad_chi_dev || !grad_us_dev || !grad_xw_dev) return fail(c, PS_EINVAL, "ps_mask_nodes_vjp: null argument");
    if (!c->has_last_mask)
        return fail(c, PS_ESTATE, "ps_mask_nodes_vjp: the current mask did not come from ps_set_mask_from_nodes");
    DeviceGuard dg(c->device);
    const MaskArgs& a = c->last_mask;
    MaskWs m = mask_ws_split(c->mask_ws, c->p.n, c->p.nz);
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->gX, 0, (size_t)a.n_nodes * 3 * sizeof(double), c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "ps_mask_nodes_vjp");
    if (a.profile == PS_MASK_TANH) {
        if (c->fp64) k_mask_vjp_dense<double><<<16 * kRasterSM, 128, 0, c->stream>>>(m, a, (const double*)grad_chi_dev, (const double*)grad_us_dev, (const double*)c->b.chi, c->gX);
        else k_mask_vjp_dense<float><<<16 * kRasterSM, 128, 0, c->stream>>>(m, a, (const float*)grad_chi_dev, (const float*)grad_us_dev, (const float*)c->b.chi, c->gX);
    } else {
        if (c->fp64) k_mask_vjp_list<double><<<8 * kRasterSM, 256, 0, c->stream>>>(m, a, c->mask_par, (const double*)grad_chi_dev, (const double*)grad_us_dev, (const double*)c->b.chi, c->gX);
        else k_mask_vjp_list<float><<<8 * kRasterSM, 256, 0, c->stream>>>(m, a, c->mask_par, (const float*)grad_chi_dev, (const float*)grad_us_dev, (const float*)c->b.chi, c->gX);
    }
    k_vjp_to_wing<<<(a.n_nodes + 127) / 128, 128, 0, c->stream>>>(a, c->gX, grad_xw_dev);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "ps_mask_nodes_vjp");
    return PS_OK;
}

ps_status ps_timing_enable(ps_ctx* c, int32_t on) {
    if (!c) return PS_EINVAL;
    DeviceGuard dg(c->device);
    if (on && c->tev_step.empty()) {
        c->tev_step.resize((size_t)kTimingRing * kEvPerStep);
        c->tev_mask.resize((size_t)kTimingRing * 2);
        for (cudaEvent_t& ev : c->tev_step)
            if (cudaEventCreate(&ev) != cudaSuccess) return fail(c, PS_ECUDA, "ps_timing_enable: cudaEventCreate");
        for (cudaEvent_t& ev : c->tev_mask)
            if (cudaEventCreate(&ev) != cudaSuccess) return fail(c, PS_ECUDA, "ps_timing_enable: cudaEventCreate");
    }
    c->timing = on != 0;
    c->t_steps = 0;
    c->t_masks = 0;
    return PS_OK;
}

ps_status ps_timing_read(ps_ctx* c, double* ms, int64_t* launches, int32_t cap, int32_t* count) {
    if (!c || !count) return PS_EINVAL;
    const int np = 6;
    *count = np;
    if (!ms || !launches || cap < np) return PS_OK;
    DeviceGuard dg(c->device);
    ps_status s = sync(c, "ps_timing_read");
    if (s != PS_OK) return s;
    for (int i = 0; i < np; ++i) { ms[i] = 0.0; launches[i] = 0; }
    const long ns = c->t_steps < kTimingRing ? c->t_steps : kTimingRing;
    auto el = [&](cudaEvent_t a0, cudaEvent_t a1, double* acc) -> bool {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, a0, a1) != cudaSuccess) return false;
        *acc += t;
        return true;
    };
    for (long k = 0; k < ns; ++k) {
        cudaEvent_t* ev = &c->tev_step[(size_t)k * kEvPerStep];
        bool ok = true;
        for (int i = 0; i < 5 && ok; ++i) ok = el(ev[2 * i], ev[2 * i + 1], &ms[i]);
        if (!ok) return fail(c, PS_ECUDA, "ps_timing_read");
        for (int i = 0; i < 5; ++i) launches[i] += 1;
    }
    const long nm = c->t_masks < kTimingRing ? c->t_masks : kTimingRing;
    for (long k = 0; k < nm; ++k) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, c->tev_mask[(size_t)k * 2], c->tev_mask[(size_t)k * 2 + 1]) != cudaSuccess)
            return fail(c, PS_ECUDA, "ps_timing_read");
        ms[5] += t;
        launches[5] += 1;
    }
    return PS_OK;
}

const char* ps_timing_name(int32_t i) { return (i >= 0 && i < 6) ? kPassNames[i] : ""; }

const char* ps_last_error(const ps_ctx* c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
