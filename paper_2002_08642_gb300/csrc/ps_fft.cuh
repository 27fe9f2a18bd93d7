// ps_fft.cuh -- in-register small DFTs and a shared-memory Stockham FFT of a
// tile of independent length-N lines, the building block of every transform
// pass of the pseudo-spectral step (Sec. 4.1, "Fourier pseudospectral
// discretization").
//
// Transform convention: X_m = sum_j x_j exp(SIGN * 2 pi i m j / N), no scaling.
//
// A length-N line (N = 2^a 3^b) is done in S radix stages: radix 16 while
// the power-of-two part allows, then its leftover (2, 4 or 8), then radix 3.
// Stage s of radix r, with Ls = product of the earlier radices, takes for
// each butterfly j in [0, N/r) the inputs x[j + t N/r] (t < r), multiplies
// input t by w^(t k) with k = j mod Ls and w = exp(SIGN 2 pi i / (Ls r)),
// does an r-point DFT in registers and writes output u to
// y[(j - k) r + k + u Ls] (Stockham order; the last stage leaves natural
// order). The first stage may read through a caller functor (global memory,
// with any pointwise operation fused in) and the last stage may write through
// one, so a line costs one shared-memory round trip per stage boundary.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ps {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx = typename cplx_of<T>::type;

template <typename C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

template <typename C, typename R> __host__ __device__ __forceinline__ C cmk(R a, R b) {
    C r; r.x = a; r.y = b; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmk<C>(a.x, -a.y); }

// FP32 complex add and subtract as one packed two-lane instruction each
// (sm_100 and later execute a float2 add as a single f32x2 operation; each
// lane is rounded like the scalar add, so results are unchanged).
#ifndef PS_F32X2
#define PS_F32X2 1
#endif
#if PS_F32X2
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
#endif
// a * (SIGN i)
template <int SIGN, typename C> __device__ __forceinline__ C rot_i(C a) {
    if constexpr (SIGN > 0) return cmk<C>(-a.y, a.x);
    else return cmk<C>(a.y, -a.x);
}

// cos and sin of 2 pi e / 16 (exact algebraic values).
__host__ __device__ constexpr double tw16_cos(int e) {
    constexpr double c1 = 0.92387953251128675613;  // cos(pi/8)
    constexpr double s1 = 0.38268343236508977173;  // sin(pi/8)
    constexpr double r2 = 0.70710678118654752440;  // sqrt(1/2)
    const int q = ((e % 16) + 16) % 16;
    return q == 0 ? 1.0 : q == 1 ? c1 : q == 2 ? r2 : q == 3 ? s1 : q == 4 ? 0.0 : q == 5 ? -s1
         : q == 6 ? -r2 : q == 7 ? -c1 : q == 8 ? -1.0 : q == 9 ? -c1 : q == 10 ? -r2
         : q == 11 ? -s1 : q == 12 ? 0.0 : q == 13 ? s1 : q == 14 ? r2 : c1;
}
__host__ __device__ constexpr double tw16_sin(int e) { return tw16_cos(e - 4); }

// a * exp(SIGN 2 pi i e / R), R | 16; e is a compile-time constant after
// unrolling, so the branches and constants fold away.
template <int R, int SIGN, typename C> __device__ __forceinline__ C twc(C a, int e) {
    using T = typename real_of<C>::type;
    const int q = ((e * (16 / R)) % 16 + 16) % 16;
    if (q == 0) return a;
    if (q == 4) return rot_i<SIGN>(a);
    if (q == 8) return cmk<C>(-a.x, -a.y);
    if (q == 12) return rot_i<-SIGN>(a);
    const T c = (T)tw16_cos(q);
    const T s = (T)(SIGN * tw16_sin(q));
    return cmk<C>(a.x * c - a.y * s, a.x * s + a.y * c);
}

// In-register DFT of R points, natural order in and out.
template <int R, int SIGN, typename C> struct Dft;

template <int SIGN, typename C> struct Dft<1, SIGN, C> {
    static __device__ __forceinline__ void run(C*) {}
};

template <int SIGN, typename C> struct Dft<2, SIGN, C> {
    static __device__ __forceinline__ void run(C* x) {
        C a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[1] = csub(a, b);
    }
};

template <int SIGN, typename C> struct Dft<3, SIGN, C> {
    static __device__ __forceinline__ void run(C* x) {
        using T = typename real_of<C>::type;
        const T h = (T)0.86602540378443864676;  // sin(2 pi / 3)
        C s = cadd(x[1], x[2]);
        C d = csub(x[1], x[2]);
        C m = cmk<C>(x[0].x - (T)0.5 * s.x, x[0].y - (T)0.5 * s.y);
        C r = rot_i<SIGN>(cmk<C>(d.x * h, d.y * h));
        x[0] = cadd(x[0], s);
        x[1] = cadd(m, r);
        x[2] = csub(m, r);
    }
};

template <int SIGN, typename C> struct Dft<4, SIGN, C> {
    static __device__ __forceinline__ void run(C* x) {
        C a = cadd(x[0], x[2]), b = csub(x[0], x[2]);
        C c = cadd(x[1], x[3]), d = rot_i<SIGN>(csub(x[1], x[3]));
        x[0] = cadd(a, c);
        x[2] = csub(a, c);
        x[1] = cadd(b, d);
        x[3] = csub(b, d);
    }
};

// R = P Q in registers: input n = Q n1 + n2, output k = k1 + P k2.
template <int P, int Q, int SIGN, typename C> __device__ __forceinline__ void dft_pq(C* x) {
    C y[P * Q];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) {
        C t[P];
#pragma unroll
        for (int n1 = 0; n1 < P; ++n1) t[n1] = x[Q * n1 + n2];
        Dft<P, SIGN, C>::run(t);
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) y[n2 * P + k1] = twc<P * Q, SIGN>(t[k1], n2 * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
        C t[Q];
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) t[n2] = y[n2 * P + k1];
        Dft<Q, SIGN, C>::run(t);
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) x[k1 + P * k2] = t[k2];
    }
}

template <int SIGN, typename C> struct Dft<8, SIGN, C> {
    static __device__ __forceinline__ void run(C* x) { dft_pq<2, 4, SIGN>(x); }
};
template <int SIGN, typename C> struct Dft<16, SIGN, C> {
    static __device__ __forceinline__ void run(C* x) { dft_pq<4, 4, SIGN>(x); }
};

// ---------------------------------------------------------------- radix plan
__host__ __device__ constexpr int pow2_part(int n) {
    int p = 1;
    while (n > 0 && n % 2 == 0) { n /= 2; p *= 2; }
    return p;
}
__host__ __device__ constexpr int n_stages(int n) {
    int p = pow2_part(n), s = 0;
    while (p >= 16) { p /= 16; ++s; }
    if (p > 1) ++s;
    int q = n / pow2_part(n);
    while (q > 1) { q /= 3; ++s; }
    return s;
}
__host__ __device__ constexpr int radix_at(int n, int s) {
    int p = pow2_part(n), i = 0;
    while (p >= 16) { if (i == s) return 16; p /= 16; ++i; }
    if (p > 1) { if (i == s) return p; ++i; }
    return 3;
}
__host__ __device__ constexpr int ls_at(int n, int s) {
    int l = 1;
    for (int i = 0; i < s; ++i) l *= radix_at(n, i);
    return l;
}
// offset of stage s's twiddle block: stages s >= 1 keep (r - 1) Ls entries,
// entry (t - 1) Ls + k = exp(+2 pi i t k / (Ls r)); the total is n - radix_at(n, 0).
__host__ __device__ constexpr int tw_offset(int n, int s) {
    int o = 0;
    for (int i = 1; i < s; ++i) o += (radix_at(n, i) - 1) * ls_at(n, i);
    return o;
}
__host__ __device__ constexpr int tw_count(int n) { return n - radix_at(n, 0); }
__host__ __device__ constexpr bool size_ok(int n) {
    int m = n;
    while (m % 2 == 0) m /= 2;
    while (m % 3 == 0) m /= 3;
    return m == 1 && n >= 4 && n % 2 == 0;
}

// ----------------------------------------------------------- line transform
// Tile address of a line stored with one padding element after every 16
// (no bank conflicts for 16-element strides): base + p + p/16. Since
// (a + 16 m) + (a + 16 m)/16 = pad(a) + 17 m for every a, a stage whose
// input stride or output stride is a multiple of 16 addresses its elements
// as a per-butterfly base plus compile-time offsets.
struct Pad16 {
    int base;
    __device__ __forceinline__ int operator()(int p) const { return base + p + (p >> 4); }
};
template <class A> struct is_pad16 { static constexpr bool value = false; };
template <> struct is_pad16<Pad16> { static constexpr bool value = true; };

// Mask of this warp's lanes that exist (the block's last warp may be partial).
__device__ __forceinline__ unsigned warp_lanes() {
    const int left = (int)blockDim.x - (int)(threadIdx.x & ~31u);
    return left >= 32 ? 0xffffffffu : ((1u << left) - 1u);
}

// One length-N line per thread group of G = N / R0 threads. `addr(p)` maps
// line position p to this thread's shared-memory slot of the tile; `load(p)`
// feeds the first stage when FROM_TILE is false; `store(p, v)` receives the
// last stage's outputs (natural order). The caller must __syncthreads()
// before the call if the tile was in use; stage boundaries sync internally,
// so every thread of the block must make the call. WS: every line's G
// threads lie in one warp and touch only their own line's slots, so a warp
// barrier separates the stages instead of a block barrier.
template <typename T, int N, int SIGN, bool WS = false> struct LineFFT {
    using C = cplx<T>;
    static constexpr int S = n_stages(N);
    static constexpr int R0 = radix_at(N, 0);
    static constexpr int G = N / R0;
    // last stage: radix, butterflies per thread; SLOTS outputs per thread
    static constexpr int RL = radix_at(N, S - 1);
    static constexpr int NBL = (N / RL + G - 1) / G;
    static constexpr int SLOTS = NBL * RL;
    static_assert(!WS || (G <= 32 && 32 % G == 0), "warp-synchronous lines must not cross warps");

    // stage barrier; lanes = the warp's lanes taking part (WS only)
    static __device__ __forceinline__ void sync(unsigned lanes) {
        if constexpr (WS) __syncwarp(lanes);
        else __syncthreads();
    }

    // BU: the last stage calls store(slot, position, value) with the
    // compile-time slot b * RL + u (butterfly b, output u), so a caller can
    // keep a thread's outputs in registers; otherwise store(position, value).
    struct NoHook {
        __device__ __forceinline__ void operator()() const {}
    };
    // TS: the last stage writes its outputs back into the tile, in place
    // (store is not called).
    template <int s, bool FROM_TILE, bool BU = false, bool TS = false, class Addr, class Load, class Store,
              class Hook = NoHook>
    static __device__ __forceinline__ void stage(C* tile, const C* tw, const Addr& addr, int g,
                                                 const Load& load, const Store& store, bool on, unsigned lanes,
                                                 const Hook& hook = Hook()) {
        constexpr int r = radix_at(N, s);
        constexpr int Ls = ls_at(N, s);
        constexpr int NBF = N / r;
        constexpr int NB = (NBF + G - 1) / G;
        constexpr bool last = (s == S - 1);
        constexpr bool from_tile = (s > 0) || FROM_TILE;
        constexpr int two = tw_offset(N, s);
        constexpr bool pad = is_pad16<Addr>::value;
        // one butterfly: inputs, twiddles, DFT
        auto gather = [&](int j, C* v) {
            const int k = j % Ls;
#pragma unroll
            for (int t = 0; t < r; ++t) {
                C x;
                if constexpr (from_tile) {
                    if constexpr (pad && NBF % 16 == 0) x = tile[addr(j) + t * (NBF + NBF / 16)];
                    else x = tile[addr(j + t * NBF)];
                } else {
                    x = load(j + t * NBF);
                }
                if constexpr (Ls > 1) {
                    if (t > 0) {
                        C w = tw[two + (t - 1) * Ls + k];
                        if constexpr (SIGN < 0) w.y = -w.y;
                        x = cmul(x, w);
                    }
                }
                v[t] = x;
            }
        };
        auto scatter = [&](int j, C* v, int b) {
            const int k = j % Ls;
            Dft<r, SIGN, C>::run(v);
#pragma unroll
            for (int u = 0; u < r; ++u) {
                const int o = (j - k) * r + k + u * Ls;
                if constexpr (last && !TS) {
                    if constexpr (BU) store(b * r + u, o, v[u]);
                    else store(o, v[u]);
                } else if constexpr (pad && Ls % 16 == 0) {
                    tile[addr((j - k) * r + k) + u * (Ls + Ls / 16)] = v[u];
                } else if constexpr (pad && Ls == 1 && r == 16) {
                    tile[addr(16 * j) + u] = v[u];
                } else {
                    tile[addr(o)] = v[u];
                }
            }
        };
        if constexpr (from_tile && !last) {
            // in place: every read of the stage before any write
            C v[NB][r];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int j = g + b * G;
                if (on && (NB * G == NBF || j < NBF)) gather(j, v[b]);
            }
            sync(lanes);
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int j = g + b * G;
                if (on && (NB * G == NBF || j < NBF)) scatter(j, v[b], b);
            }
        } else if constexpr (BU && last) {
            // one butterfly at a time, unrolled so that slots are constants
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int j = g + b * G;
                if (on && (NB * G == NBF || j < NBF)) {
                    C v[r];
                    gather(j, v);
                    scatter(j, v, b);
                }
            }
        } else {
            // reads from the functor, or the last stage (each butterfly reads
            // and writes the same positions): one butterfly at a time
#pragma unroll 1
            for (int b = 0; b < NB; ++b) {
                const int j = g + b * G;
                if (on && (NB * G == NBF || j < NBF)) {
                    C v[r];
                    gather(j, v);
                    scatter(j, v, b);
                }
            }
        }
        if constexpr (!last) sync(lanes);
        if constexpr (s == 0 && !last) hook();
        if constexpr (s + 1 < S) stage<s + 1, FROM_TILE, BU, TS>(tile, tw, addr, g, load, store, on, lanes, hook);
    }

    template <bool FROM_TILE, class Addr, class Load, class Store>
    static __device__ __forceinline__ void run(C* tile, const C* tw, const Addr& addr, int g,
                                               const Load& load, const Store& store) {
        stage<0, FROM_TILE>(tile, tw, addr, g, load, store, true, WS ? warp_lanes() : 0u);
    }
    // Same, and hook() is called by every thread right after the barrier
    // that ends the first stage (every load() call done); a one-stage
    // transform (S == 1) has no such barrier and never calls it.
    template <bool FROM_TILE, class Addr, class Load, class Store, class Hook>
    static __device__ __forceinline__ void run_hook(C* tile, const C* tw, const Addr& addr, int g,
                                                    const Load& load, const Store& store, const Hook& hook) {
        stage<0, FROM_TILE, false>(tile, tw, addr, g, load, store, true, WS ? warp_lanes() : 0u, hook);
    }
    // Last-stage outputs delivered as store(slot, position, value).
    template <bool FROM_TILE, class Addr, class Load, class Store>
    static __device__ __forceinline__ void run_bu(C* tile, const C* tw, const Addr& addr, int g,
                                                  const Load& load, const Store& store) {
        stage<0, FROM_TILE, true>(tile, tw, addr, g, load, store, true, WS ? warp_lanes() : 0u);
    }
    // Outputs written back into the tile (natural order, in place).
    template <bool FROM_TILE, class Addr, class Load>
    static __device__ __forceinline__ void run_tile(C* tile, const C* tw, const Addr& addr, int g,
                                                    const Load& load) {
        auto nostore = [](int, C) {};
        stage<0, FROM_TILE, false, true>(tile, tw, addr, g, load, nostore, true, WS ? warp_lanes() : 0u);
    }
    // Same, for the threads with on == true (see run_masked).
    template <bool FROM_TILE, class Addr, class Load>
    static __device__ __forceinline__ void run_tile_masked(C* tile, const C* tw, const Addr& addr, int g,
                                                           const Load& load, bool on) {
        auto nostore = [](int, C) {};
        if constexpr (WS) {
            const unsigned lanes = __ballot_sync(warp_lanes(), on);
            if (!on) return;
            stage<0, FROM_TILE, false, true>(tile, tw, addr, g, load, nostore, true, lanes);
        } else {
            stage<0, FROM_TILE, false, true>(tile, tw, addr, g, load, nostore, on, 0u);
        }
    }
    // Same, for the threads with on == true. Block barriers: the others
    // still take part in them. Warp barriers (WS): the others leave at once
    // (on must be the same for all G threads of a line).
    template <bool FROM_TILE, class Addr, class Load, class Store>
    static __device__ __forceinline__ void run_masked(C* tile, const C* tw, const Addr& addr, int g,
                                                      const Load& load, const Store& store, bool on) {
        if constexpr (WS) {
            const unsigned lanes = __ballot_sync(warp_lanes(), on);
            if (!on) return;
            stage<0, FROM_TILE>(tile, tw, addr, g, load, store, true, lanes);
        } else {
            stage<0, FROM_TILE>(tile, tw, addr, g, load, store, on, 0u);
        }
    }
};

}  // namespace ps
