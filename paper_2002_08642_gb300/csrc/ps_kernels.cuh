// ps_kernels.cuh -- the transform passes and fused pointwise kernels of one
// time step of the penalized pseudo-spectral Navier--Stokes solver
// (Sec. 4.1, Eq. penalized Navier--Stokes; time stepping paragraph).
//
// Storage (element = complex T unless stated):
//   U, H   spectral velocity c_k = DFT(u)_k / n^3 and AB2 history
//          Q^n = E U^n - (dt/2) E^2 N^{n-1} (see ab2_update),
//          3 x [K (ky)][K (kx)][Kzp] (an x line of fixed ky, kz is a
//          contiguous block), only the modes the 2/3 rule keeps:
//          x/y index c in [0, K) <-> mode m = c (c <= mmax) or c - K,
//          z index c in [0, Kz) <-> mode m = c; K = 2 mmax + 1, Kz = mmax + 1,
//          mmax = (n - 1) / 3, Kzp = Kz rounded up to the tile width.
//   A      after the x transform: nf x [K][n][Kzp]   (y spectral, x physical,
//          z spectral; also the y-forward output read by the x-forward pass).
//          x lines of fixed ky are contiguous, so an x-pass tile stays within
//          one n Kzp block; with x outermost instead, the x-inverse's stores
//          of one tile spread over the whole field and it ran 1.6x slower at
//          n = 768 (the y passes, whose tiles then stride by n Kzp per row,
//          measured the same either way).
//   B      after the y transform: nf x [n][n][Kzp]   (x/y physical, z spectral)
//   chi    n^3 real, us 3 x n^3 real, line flag [n][n] (1 if the z line
//          touches chi > 0)
// Every aliased mode is identically zero, so the passes never read or write
// it: the x pass reads K of n rows, the y pass K of n rows, and the z pass
// Kz of n/2+1 entries per line.
//
// Pass order of a step (P = Leray projection, E = exp(-nu |k|^2 dt)); the
// step uses the TMA-staged kernels k_xinv_tma, k_yinv_tma, k_zpass,
// k_yfwd_tma, k_xfwd_tma; the plain kernels k_xinv/k_yinv/k_yfwd/k_xfwd and
// the physical <-> z-spectral kernels serve ps_set/get_velocity and the
// adjoint's generic transforms:
//   1 x-inverse of u_hat and omega_hat = i k x u_hat (curl fused)    U -> A (6)
//   2 y-inverse                                                      A -> B (6)
//   3 z c2r, n = u x omega - (chi/eta)(u - u_s), force/moment partial
//     sums in double, z r2c truncated to Kz                          B -> B (3)
//   4 y-forward truncated to K rows                                  B -> A (3)
//   5 x-forward truncated to K rows, 1/n^3, P, integrating-factor
//     AB2 (Euler on the first step)                                  A,U,H -> U,H
#pragma once
// launch-shape knobs of the z pass (threads per block cap, shared memory
// cap in KiB, blocks per SM the register budget is sized for)
#ifndef PS_ZP_MAXTHR
#define PS_ZP_MAXTHR 384
#endif
#ifndef PS_ZP_SMEM_KB
#define PS_ZP_SMEM_KB 100
#endif
#ifndef PS_ZP_MINB
#define PS_ZP_MINB 0   // 0: automatic (Geo::ZMINB)
#endif
// z-pass staging buffers: 2 = the next batch's copy overlaps the whole
// batch; 1 = it is issued once the inverse transforms have read the buffer
#ifndef PS_ZP_NBUF
#define PS_ZP_NBUF 1
#endif
// 1: z lines of n = 3M done as three length-M transforms (see k_zpass)
#ifndef PS_Z3
#define PS_Z3 1
#endif
// 1: z-pass line transforms whose threads fit in one warp sync by warp
#ifndef PS_ZWS
#define PS_ZWS 1
#endif
// tile width of the TMA-staged y passes (0 = automatic)
#ifndef PS_TY_C
#define PS_TY_C 0
#endif
// y-inverse staging buffers: 2 = the next item's copy overlaps the whole
// item; 1 = it is issued once the first FFT stage has read the buffer
#ifndef PS_Y2_NBUF
#define PS_Y2_NBUF 1
#endif
#ifndef PS_Y2_SMEM_KB
#define PS_Y2_SMEM_KB 226
#endif
#ifndef PS_Y4_SMEM_KB
#define PS_Y4_SMEM_KB 226
#endif
#ifndef PS_X1_SMEM_KB
#define PS_X1_SMEM_KB 64
#endif
#ifndef PS_X5_SMEM_KB
#define PS_X5_SMEM_KB 200
#endif

#include "ps_async.cuh"
#include "ps_fft.cuh"

namespace ps {

struct KP {
    int n, nz;        // points along x and y (n), along z (nz: n, or n/2 for the 4 x 4 x 2 box)
    int mmax, K, Kz, Kzp;   // mmax, K from n; Kz = (nz - 1)/3 + 1 kept z modes, Kzp padded
    double ks;        // 2 pi / L
    double ksz;       // 2 pi / Lz (Lz = L nz / n: the same spacing on every axis)
    double dt, inv_eta, invn3, dx, half_L3;
    double x0[3];
    int mean_free;
    int xs0, xsn;     // x planes [xs0, xs0 + xsn) handled by the y and z passes
    int ky0, kyn;     // kept ky rows [ky0, ky0 + kyn) handled by the TMA x passes (slab decomposition)
    int part_off;     // first force-partial slot of this z-pass launch
    double inv_csp;   // 1 / C_sp of the sponge term (used by the sponge variants only)
};

__device__ __forceinline__ int mode_of(int q, int n) { return q < n / 2 ? q : q - n; }
__device__ __forceinline__ int cidx_of(int m, int K) { return m >= 0 ? m : m + K; }
__device__ __forceinline__ int cmode_of(int c, int mmax, int K) { return c <= mmax ? c : c - K; }

// Neumaier-compensated accumulation in double.
struct Acc {
    double s, c;
    __device__ __forceinline__ void add(double v) {
        double t = s + v;
        if (fabs(s) >= fabs(v)) c += (s - t) + v;
        else c += (v - t) + s;
        s = t;
    }
    __device__ __forceinline__ double val() const { return s + c; }
};

// Block-wide sum of `nv` doubles per thread into out[0..nv) (thread 0 writes).
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* out, double* scratch) {
    for (int i = 0; i < NV; ++i) {
        double x = v[i];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        v[i] = x;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0)
        for (int i = 0; i < NV; ++i) scratch[wid * NV + i] = v[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < NV; ++i) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += scratch[w * NV + i];
            out[i] = s;
        }
    }
}

// Launch geometry per (T, n): tile width C of the strided passes (128-byte
// rows), C5 of the x-forward/update pass (three tiles must fit), the z
// pass's lines per batch and the TMA passes' tile widths.
template <typename T, int N> struct Geo {
    using C2 = cplx<T>;
    static constexpr int G = LineFFT<T, N, 1>::G;
    static constexpr int CW = 128 / (int)sizeof(C2);     // 16 (float), 8 (double)
    static constexpr int C = CW;
    static constexpr int C5 = (3 * N * CW * (int)sizeof(C2) <= 110 * 1024) ? CW
                            : (3 * N * (CW / 2) * (int)sizeof(C2) <= 150 * 1024) ? CW / 2 : CW / 4;
    static constexpr int LP = N + N / 16;                  // padded z line
    // kept z modes, padded to the tile width
    static constexpr int KZ = (N - 1) / 3 + 1;
    static constexpr int KZP = (KZ + CW - 1) / CW * CW;
    // z pass: LZ lines per batch (even, divides n^2), 3 LZ G threads,
    // ZNB staging buffers of the batch's six spectral lines plus the FFT tiles
    static constexpr int ZNB = PS_ZP_NBUF == 1 ? 1 : 2;
    static constexpr int zsmem(int l) {
        return (int)sizeof(C2) * (ZNB * 6 * l * KZP + 3 * l * LP + tw_count(N) + 1) + 128;
    }
    // lines of at most 16 threads take batches of 2 lines (measured on GB300:
    // 256^3 z pass 0.187 -> 0.177 ms); longer lines the largest batch within
    // the thread and shared-memory budgets (384^3: 0.611 ms against 0.652 ms
    // with 2 lines)
    static constexpr int lz_pick() {
        const int maxthr = G <= 16 ? 6 * G : PS_ZP_MAXTHR;
        int l = 2;
        while (3 * (2 * l) * G <= maxthr && zsmem(2 * l) <= PS_ZP_SMEM_KB * 1024 && (N * N) % (2 * l) == 0)
            l *= 2;
        return l;
    }
    static constexpr int LZ = lz_pick();
    // three blocks per SM where the register cap this sets (<= 72 at 288
    // threads) costs no more than a few spilled words, else two; never more
    // than the shared memory lets reside
    static constexpr int ZFIT = (227 * 1024) / (zsmem(LZ) + 4096) > 0 ? (227 * 1024) / (zsmem(LZ) + 4096) : 1;
    static constexpr int ZMIN0 = (3 * LZ * G <= 288 || N <= 256) ? 3 : 2;
    static constexpr int ZMINB = PS_ZP_MINB > 0 ? PS_ZP_MINB : (ZMIN0 < ZFIT ? ZMIN0 : ZFIT);
    // TMA-staged y passes: K = kept x/y modes; inputs come in boxes of at
    // most 256 rows (NBOX boxes of BR rows cover R rows)
    static constexpr int K = 2 * ((N - 1) / 3) + 1;
    static constexpr int nbox(int r) { return (r + 255) / 256; }
    static constexpr int brows(int r) { return (r + nbox(r) - 1) / nbox(r); }
    // row of (x, ky) within a field of A: [ky][x], an x line is contiguous
    static __host__ __device__ constexpr size_t arow(int x, int ky) { return (size_t)ky * N + x; }
    // smem rows between box starts: every box lands 128-byte aligned
    static constexpr int bpitch(int r, int c) {
        const int q = 128 / (c * (int)sizeof(C2)) > 0 ? 128 / (c * (int)sizeof(C2)) : 1;
        return (brows(r) + q - 1) / q * q;
    }
    static constexpr int Y2NB = PS_Y2_NBUF == 1 ? 1 : 2;
    static constexpr int y2_smem(int c, int nb = 2) {   // y inverse: nb staging (K rows) + work tile (N rows)
        return (int)sizeof(C2) * c * (nb * nbox(K) * bpitch(K, c) + N) + (int)sizeof(C2) * (tw_count(N) + 1) + 256;
    }
    static constexpr int y4_smem(int c) {   // y forward: 2 staging tiles of N rows, transformed in place
        return (int)sizeof(C2) * c * (2 * nbox(N) * bpitch(N, c)) + (int)sizeof(C2) * (tw_count(N) + 1) + 256;
    }
    static constexpr int x5_smem(int c, int nf = 3) {   // x forward: 2 staging tiles (N rows) + nf result tiles
        return (int)sizeof(C2) * c * (2 * nbox(N) * bpitch(N, c) + nf * K) + (int)sizeof(C2) * (tw_count(N) + 1) + 256;
    }
    // widest tile (at most cmax complex, at least 2) whose shared memory fits
    static constexpr int pick_c(int which, int kb, int cmax) {
        if (PS_TY_C > 0) return PS_TY_C;
        int c = cmax < CW ? cmax : CW;
        while (c > 2 && (which == 1 ? y2_smem(c) : which == 2 ? y2_smem(c, Y2NB) : which == 4 ? y4_smem(c) : x5_smem(c)) >
                            kb * 1024)
            c /= 2;
        return c;
    }
    // budgets measured on GB300 (FP32 and FP64 alike): the y passes and the
    // x-forward pass prefer one wide tile per SM, the x-inverse (two register
    // sets of outputs per thread) several narrow ones
    static constexpr int CY2 = pick_c(2, PS_Y2_SMEM_KB, 16);
    static constexpr int CY4 = pick_c(4, PS_Y4_SMEM_KB, 16);
    static constexpr int CX1 = pick_c(1, PS_X1_SMEM_KB, 16);   // same smem shape as the y inverse, two buffers
    static constexpr int CX5 = pick_c(5, PS_X5_SMEM_KB, 128 / 16);
    static constexpr int tw_n = tw_count(N) > 0 ? tw_count(N) : 1;
};

__device__ __forceinline__ int zaddr(int p, int line, int LP) { return line * LP + p + (p >> 4); }

// Physical <-> z-spectral transforms (k_zinv_phys, k_zfwd_phys): persistent
// blocks over batches of L lines (L even, dividing n^2), three thread groups
// of G threads per line pair, one transform each: (u_x + i u_y) of either
// line and (u_z[2m] + i u_z[2m + 1]). A batch's three fields come by bulk
// copies into one of two staging buffers (spectral: L Kzp complex per field;
// physical: L N reals per field). L is the batch that puts the most threads
// on an SM within the shared memory.
template <typename T, int N> struct ZPhys {
    using C2 = cplx<T>;
    static constexpr int G = LineFFT<T, N, 1>::G;
    static constexpr int LP = N + N / 16;
    static constexpr int KZP = Geo<T, N>::KZP;
    static constexpr int TWN = Geo<T, N>::tw_n;
    static constexpr int smem(int l, bool fwd) {
        const int stage = fwd ? 2 * 3 * l * N * (int)sizeof(T) : 2 * 3 * l * KZP * (int)sizeof(C2);
        return stage + (int)sizeof(C2) * (3 * (l / 2) * LP + TWN) + 128;
    }
    static constexpr int threads(int l) { return 3 * (l / 2) * G; }
    static constexpr int resident(int l, bool fwd) {   // threads per SM
        int b = (227 * 1024) / (smem(l, fwd) + 1024);
        if (b * threads(l) > 2048) b = 2048 / threads(l);
        if (b > 32) b = 32;
        return b * threads(l);
    }
    static constexpr int pick(bool fwd) {
        int best = 2;
        for (int l = 4; l <= 8; l *= 2)
            if (threads(l) <= 512 && resident(l, fwd) >= resident(best, fwd)) best = l;
        return best;
    }
    static constexpr int LI = pick(false), LF = pick(true);
    // k_zinv_sub: one field, one thread group per line pair; a batch stages
    // its L spectral lines and its L physical lines of u
    static constexpr int smem_sub(int l) {
        return 2 * l * (KZP * (int)sizeof(C2) + N * (int)sizeof(T)) + (int)sizeof(C2) * ((l / 2) * LP + TWN) + 128;
    }
    static constexpr int threads_sub(int l) { return (l / 2) * G; }
    static constexpr int resident_sub(int l) {
        int b = (227 * 1024) / (smem_sub(l) + 1024);
        if (b * threads_sub(l) > 2048) b = 2048 / threads_sub(l);
        if (b > 32) b = 32;
        return b * threads_sub(l);
    }
    static constexpr int pick_sub() {
        int best = 2;
        for (int l = 4; l <= 16; l *= 2)
            if (threads_sub(l) <= 512 && resident_sub(l) >= resident_sub(best)) best = l;
        return best;
    }
    static constexpr int LS = pick_sub();
};

// Dynamic shared memory rounded up to a 128-byte boundary (TMA destinations
// need it; kernels reserve 128 bytes of slack). The extern array's own
// alignment is not relied on.
__device__ __forceinline__ unsigned char* smem_base128(unsigned char* raw) {
    const uint32_t a = smem_u32(raw);
    return raw + ((128u - (a & 127u)) & 127u);
}

// ----------------------------------------------- n = 3M split of a line
// With the 2/3 rule and n = 3M, a line's kept modes are q in [0, M) and
// (2M, 3M): the middle third is empty. The inverse transform then is three
// length-M transforms, z[3a + b] = sum_q e^{2 pi i a q / M} Y_b[q],
//   Y_b[q] = e^{2 pi i b q / n} (X[q] + e^{2 pi i 2b/3} X[q + 2M]),
// and the forward transform's kept outputs come from the length-M
// transforms F_b of z[3a + b]:
//   Z[k] = sum_b e^{-2 pi i b k/n} F_b[k],
//   Z[2M + k] = sum_b e^{-2 pi i 2b/3} e^{-2 pi i b k/n} F_b[k].
// tw3[(b - 1) M + q] = e^{+2 pi i b q / n} (b = 1, 2).
// The z pass uses both directions; the TMA x and y passes use the forward
// one (split3_out). Their inverses keep the length-n transform: the split's
// two-mode input loads and per-sub-line register sets cost more there than
// the stage it saves.
template <typename T, int N> struct Split3 {
    static constexpr bool on = (N % 3 == 0) && (PS_Z3 != 0);
    static constexpr int M = on ? N / 3 : N;
    static constexpr int GM = LineFFT<T, M, 1>::G;                     // threads per sub-line
    static constexpr int TWM = on ? (tw_count(M) > 0 ? tw_count(M) : 1) : 0;
    // the block's thread groups split evenly over the three sub-lines, and
    // the M table plus tw3 fit in the room of the n table (+ 1)
    static_assert(!on || 3 * GM == LineFFT<T, N, 1>::G, "n = 3M split: group count");
    static_assert(!on || TWM + 2 * M <= tw_count(N) + 1, "n = 3M split: twiddle room");
};

// Z[k] and Z[2M + k] from F_0[k], F_1[k], F_2[k].
template <typename C2>
__device__ __forceinline__ void split3_out(C2 F0, C2 F1, C2 F2, const C2* tw3, int k, int M, C2& Zk, C2& Zm) {
    using T = typename real_of<C2>::type;
    const T h3 = (T)0.86602540378443864676;
    const C2 G1 = cmul(F1, cconj(tw3[k])), G2 = cmul(F2, cconj(tw3[M + k]));
    Zk = cadd(F0, cadd(G1, G2));
    // e^{-2 pi i 2/3} = (-1/2, +h), e^{-2 pi i 4/3} = (-1/2, -h)
    Zm = cmk<C2>(F0.x - (T)0.5 * (G1.x + G2.x) - h3 * (G1.y - G2.y),
                 F0.y - (T)0.5 * (G1.y + G2.y) + h3 * (G1.x - G2.x));
}

// The z pass's n = 3M split by mirror pairs of modes (q, m = M - q): one
// thread serves both, so each staged input and each twiddle is read once for
// all three sub-lines. Since e^{2 pi i b m / n} = e^{2 pi i b / 3}
// conj(e^{2 pi i b q / n}), the mirror needs no twiddle of its own.
// Tiles hold sub-line b at padded positions zaddr(b M + p).
//
// Inverse pre-butterfly: the input line Z = A + i B (A, B the half spectra of
// two real fields, kz < M kept) gives v = Z[q], w = Z[q + 2M] = Z[n - m],
// v' = Z[m], w' = Z[n - q], and with t_b = e^{2 pi i b q / n}:
//   Y_b[q] = t_b (v + e^{2 pi i 2b/3} w),  Y_b[m] = conj(t_b) (e^{2 pi i b/3} v' + w').
// q = 0 serves mode 0 (Z[2M] = 0; the kz = 0 inputs' imaginary parts,
// round-off of real fields, dropped) and the self-mirror mode M/2.
// Padded tile position of entry p of sub-line b (sub-lines of length M):
// zaddr(b M + p) = b (M + M/16) + zaddr(p) when 16 divides M.
template <int M>
__device__ __forceinline__ int zsub(int b, int p) {
    if constexpr (M % 16 == 0) return b * (M + M / 16) + p + (p >> 4);
    else return zaddr(b * M + p, 0, 0);
}

template <typename T, int M>
__device__ __forceinline__ void split3_pre(const cplx<T>* fa, const cplx<T>* fb, const cplx<T>* tw3, cplx<T>* t,
                                           int q) {
    using C2 = cplx<T>;
    const T h = (T)0.86602540378443864676;   // sin(2 pi / 3)
    auto put = [&](int b, int p, C2 v) { t[zsub<M>(b, p)] = v; };
    // x + e^{2 pi i 2/3} y, x + e^{-2 pi i 2/3} y  (e^{+-2 pi i 2/3} = (-1/2, -+h))
    auto rm = [&](C2 x, C2 y) { return cmk<C2>(x.x - (T)0.5 * y.x + h * y.y, x.y - (T)0.5 * y.y - h * y.x); };
    auto rp = [&](C2 x, C2 y) { return cmk<C2>(x.x - (T)0.5 * y.x - h * y.y, x.y - (T)0.5 * y.y + h * y.x); };
    constexpr int H = M / 2;
    const int qa = q == 0 ? H : q;
    const C2 a = fa[qa], c = fb[qa];
    const C2 v = cmk<C2>(a.x - c.y, a.y + c.x);    // Z[qa]
    const C2 w2 = cmk<C2>(a.x + c.y, c.x - a.y);   // Z[n - qa]
    const C2 t1 = tw3[qa], t2 = tw3[M + qa];
    if (q == 0) {
        const C2 z0 = cmk<C2>(fa[0].x, fb[0].x);
        put(0, 0, z0);
        put(1, 0, z0);
        put(2, 0, z0);
        // mode M/2: Z[M/2 + 2M] = Z[n - M/2]
        put(0, H, cadd(v, w2));
        put(1, H, cmul(rm(v, w2), t1));
        put(2, H, cmul(rp(v, w2), t2));
        return;
    }
    const int m = M - q;
    const C2 a2 = fa[m], c2 = fb[m];
    const C2 w = cmk<C2>(a2.x + c2.y, c2.x - a2.y);   // Z[q + 2M] = Z[n - m]
    const C2 v2 = cmk<C2>(a2.x - c2.y, a2.y + c2.x);  // Z[m]
    put(0, q, cadd(v, w));
    put(1, q, cmul(rm(v, w), t1));
    put(2, q, cmul(rp(v, w), t2));
    put(0, m, cadd(v2, w2));
    put(1, m, cmul(rp(w2, v2), cconj(t1)));
    put(2, m, cmul(rm(w2, v2), cconj(t2)));
}

// Forward recombination of the sub-line spectra F_b (b = 0, 1, 2) of a tile
// for the pair (k, m = M - k): with s_b = e^{2 pi i b k / n},
// G_b = conj(s_b) F_b[k], H_b = s_b F_b[m] and w = e^{2 pi i / 3},
//   Z[k] = F_0[k] + G_1 + G_2,      Z[n - m] = F_0[k] + w G_1 + w^2 G_2,
//   Z[n - k] = F_0[m] + H_1 + H_2,  Z[m] = F_0[m] + w^2 H_1 + w H_2.
// k = 0 gives Z[0] (twice) and the self-mirror mode M/2: zm = Z[M/2],
// znm = Z[n - M/2].
template <typename T, int M>
__device__ __forceinline__ void split3_pair_out(const cplx<T>* t, const cplx<T>* tw3, int k, cplx<T>& zk,
                                                cplx<T>& znk, cplx<T>& zm, cplx<T>& znm) {
    using C2 = cplx<T>;
    const T h = (T)0.86602540378443864676;
    auto at = [&](int b, int p) { return t[zsub<M>(b, p)]; };
    // x + w y + w^2 z
    auto rw = [&](C2 x, C2 y, C2 z) {
        return cmk<C2>(x.x - (T)0.5 * (y.x + z.x) - h * (y.y - z.y), x.y - (T)0.5 * (y.y + z.y) + h * (y.x - z.x));
    };
    constexpr int H = M / 2;
    const int ka = k == 0 ? H : k;
    const C2 s1 = tw3[ka], s2 = tw3[M + ka];
    const C2 f0 = at(0, ka), g1 = cmul(at(1, ka), cconj(s1)), g2 = cmul(at(2, ka), cconj(s2));
    if (k == 0) {
        zk = cadd(at(0, 0), cadd(at(1, 0), at(2, 0)));
        znk = zk;
        zm = cadd(f0, cadd(g1, g2));
        znm = rw(f0, g1, g2);
        return;
    }
    const int m = M - k;
    const C2 e0 = at(0, m), h1 = cmul(at(1, m), s1), h2 = cmul(at(2, m), s2);
    zk = cadd(f0, cadd(g1, g2));
    znm = rw(f0, g1, g2);
    znk = cadd(e0, cadd(h1, h2));
    zm = rw(e0, h2, h1);
}

// Integrating-factor AB2 update of one mode (Sec. 4.1, time stepping):
// U^{n+1} = E U^n + (dt/2)(3 E N^n - E^2 N^{n-1}). The history array holds
// Q^n = E U^n - (dt/2) E^2 N^{n-1}, the part of U^{n+1} known before N^n, so
// a step reads one array: U^{n+1} = Q^n + (3/2) dt E N^n (Euler start:
// U^1 = E (U^0 + dt N^0), reading U^0), then Q^{n+1} = E U^{n+1} - (dt/2) E^2 N^n.
// uq = Q^n (U^0 on the first step), nn = N^n.
template <typename C2, typename T>
__device__ __forceinline__ void ab2_update(C2 uq, C2 nn, T E, T dt, bool first, C2& unew, C2& qnew) {
    if (first) {
        unew = cmk<C2>(E * (uq.x + dt * nn.x), E * (uq.y + dt * nn.y));
    } else {
        const T a3 = (T)1.5 * dt * E;
        unew = cmk<C2>(uq.x + a3 * nn.x, uq.y + a3 * nn.y);
    }
    const T a2 = (T)0.5 * dt * E * E;
    qnew = cmk<C2>(E * unew.x - a2 * nn.x, E * unew.y - a2 * nn.y);
}

// Twiddles into shared memory: the n-line table, or for the n = 3M split
// the M-line table followed by tw3 (both fit in the n-line table's room).
template <typename T, int N>
__device__ __forceinline__ cplx<T>* load_tw_split(cplx<T>* tw, const cplx<T>* twg, int n_tw) {
    using S3 = Split3<T, N>;
    if constexpr (S3::on) {
        for (int i = threadIdx.x; i < tw_count(S3::M); i += blockDim.x) tw[i] = twg[N + i];
        for (int i = threadIdx.x; i < 2 * S3::M; i += blockDim.x) tw[S3::TWM + i] = twg[2 * N + i];
        return tw + S3::TWM;
    } else {
        for (int i = threadIdx.x; i < n_tw; i += blockDim.x) tw[i] = twg[i];
        return tw;
    }
}

template <typename C2>
__device__ __forceinline__ void load_tw(C2* s, const C2* g, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) s[i] = g[i];
}

// ---------------------------------------------------------------- pass 1
// x-inverse of the three velocity components and, if NF == 6, of the
// vorticity omega_hat = i k x u_hat (components 3..5).
template <typename T, int N, int NF>
__global__ void __launch_bounds__(Geo<T, N>::C * Geo<T, N>::G)
k_xinv(KP kp, const cplx<T>* __restrict__ U, cplx<T>* __restrict__ A, const cplx<T>* __restrict__ twg) {
    using C2 = cplx<T>;
    using GE = Geo<T, N>;
    constexpr int C = GE::C, G = GE::G;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* tw = reinterpret_cast<C2*>(smraw);
    C2* tile = tw + GE::tw_n;
    const int col = threadIdx.x % C, g = threadIdx.x / C;
    const int cz = blockIdx.x * C + col;
    const bool okz = cz < kp.Kz;
    const int cy = blockIdx.y;
    const int K = kp.K, mmax = kp.mmax, Kzp = kp.Kzp;
    const T ks = (T)kp.ks;   // wavenumbers in T: no double arithmetic per element
    const T ky = ks * (T)cmode_of(cy, mmax, K);
    const T kz = (T)kp.ksz * (T)cz;
    const size_t FS = (size_t)K * K * Kzp;
    const size_t AS = (size_t)N * K * Kzp;
    load_tw(tw, twg, GE::tw_n);
    auto addr = [&](int p) { return p * C + col; };
#pragma unroll 1
    for (int f = 0; f < NF; ++f) {
        __syncthreads();
        auto load = [&](int q) -> C2 {
            const int m = mode_of(q, N);
            if (!okz || m > mmax || m < -mmax) return cmk<C2>((T)0, (T)0);
            const size_t o = ((size_t)cy * K + cidx_of(m, K)) * Kzp + cz;
            const T kx = ks * (T)m;
            if (f < 3) return U[f * FS + o];
            if (f == 3) {  // i (ky uz - kz uy)
                C2 uy = U[FS + o], uz = U[2 * FS + o];
                return cmk<C2>(-(ky * uz.y - kz * uy.y), ky * uz.x - kz * uy.x);
            }
            if (f == 4) {  // i (kz ux - kx uz)
                C2 ux = U[o], uz = U[2 * FS + o];
                return cmk<C2>(-(kz * ux.y - kx * uz.y), kz * ux.x - kx * uz.x);
            }
            C2 ux = U[o], uy = U[FS + o];  // i (kx uy - ky ux)
            return cmk<C2>(-(kx * uy.y - ky * ux.y), kx * uy.x - ky * ux.x);
        };
        auto store = [&](int x, C2 v) {
            if (okz) A[f * AS + GE::arow(x, cy) * Kzp + cz] = v;
        };
        LineFFT<T, N, 1>::template run<false>(tile, tw, addr, g, load, store);
    }
}

// ---------------------------------------------------------------- pass 2
template <typename T, int N, int NF>
__global__ void __launch_bounds__(Geo<T, N>::C * Geo<T, N>::G)
k_yinv(KP kp, const cplx<T>* __restrict__ A, cplx<T>* __restrict__ B, const cplx<T>* __restrict__ twg) {
    using C2 = cplx<T>;
    using GE = Geo<T, N>;
    constexpr int C = GE::C;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* tw = reinterpret_cast<C2*>(smraw);
    C2* tile = tw + GE::tw_n;
    const int col = threadIdx.x % C, g = threadIdx.x / C;
    const int cz = blockIdx.x * C + col;
    const bool okz = cz < kp.Kz;
    const int x = blockIdx.y;
    const int K = kp.K, mmax = kp.mmax, Kzp = kp.Kzp;
    const size_t AS = (size_t)N * K * Kzp;
    const size_t BS = (size_t)N * N * Kzp;
    load_tw(tw, twg, GE::tw_n);
    auto addr = [&](int p) { return p * C + col; };
#pragma unroll 1
    for (int f = 0; f < NF; ++f) {
        __syncthreads();
        auto load = [&](int q) -> C2 {
            const int m = mode_of(q, N);
            if (!okz || m > mmax || m < -mmax) return cmk<C2>((T)0, (T)0);
            return A[f * AS + GE::arow(x, cidx_of(m, K)) * Kzp + cz];
        };
        auto store = [&](int y, C2 v) {
            if (okz) B[f * BS + ((size_t)x * N + y) * Kzp + cz] = v;
        };
        LineFFT<T, N, 1>::template run<false>(tile, tw, addr, g, load, store);
    }
}

// ---------------------------------------------------------------- pass 3
// z lines of (x, y), in batches of LZ consecutive lines, persistent blocks.
// The six spectral lines of the next batch are fetched by bulk asynchronous
// copies into the other staging buffer while the current batch is computed.
// Per line: three complex inverse transforms (u_x + i u_y, u_z + i w_x,
// w_y + i w_z) run side by side by three thread groups; n = u x omega -
// (chi/eta)(u - u_s) pointwise with the force/moment partial sums in double;
// forward transforms of (n_x + i n_y) per line and of (n_z[l] + i n_z[l+1])
// per line pair; the result, truncated to kz < Kz, overwrites fields 0..2 of
// B (only this batch's lines, whose input is already in shared memory).
//
// For n = 3M the 2/3 truncation leaves the middle third of every z spectrum
// empty (Kz = M), so a length-n line is done as three length-M transforms:
// inverse  z[3a + b] = sum_q' e^{2 pi i a q'/M} Y_b[q'],
//          Y_b[q'] = e^{2 pi i b q'/n} (Z[q'] + e^{2 pi i 2b/3} Z[q' + 2M]),
// forward  Z[k'] = sum_b e^{-2 pi i b k'/n} F_b[k'],
//          Z[2M + k'] = sum_b e^{-2 pi i 2b/3} e^{-2 pi i b k'/n} F_b[k'],
// F_b the forward length-M transform of z[3a + b]; sub-line b of a tile
// holds z[3a + b] at position b M + a, so the pointwise phase reads and
// writes in place and no reordering pass is needed. The pre-butterfly (Y_b
// into the tiles, then the inverse transforms in place) and the
// recombination (fused with the unpack to B) each go by mirror pairs of
// modes (split3_pre, split3_pair_out): every staged input, tile value and
// twiddle is read once.
// PM (pressure evaluation): also writes (1/2)|u|^2 to half_u2 (n^3,
// [x][y][z]), leaves the force partials of the last step untouched and
// writes its three result fields to Bo (Bo = B allowed), so that B can keep
// u and omega of the state for the step that follows.
// Template N is the z-line length (nz), NY the number of lines per x-plane
// and of x-planes (n; n x n x nz grid; compile time, it keeps the z pass's
// registers below the three-blocks-per-SM cap).
// SP (sponge term on): also s = chi_sp omega, transformed forward like n
// (s_x + i s_y per line by the third thread group, s_z of line pairs by the
// odd lines' second group, the groups that are otherwise idle) into B
// fields 3..5.
template <typename T, int N, bool PM = false, bool SP = false, int NY = N>
__global__ void __launch_bounds__(3 * Geo<T, N>::LZ * Geo<T, N>::G, Geo<T, N>::ZMINB)
k_zpass(KP kp, cplx<T>* __restrict__ B, const T* __restrict__ chi, const T* __restrict__ us,
        const uint8_t* __restrict__ flag, double* __restrict__ partial, const cplx<T>* __restrict__ twg,
        int* __restrict__ err, T* __restrict__ half_u2, const T* __restrict__ chi_sp, cplx<T>* Bo) {
    using C2 = cplx<T>;
    using GE = Geo<T, N>;
    constexpr int G = GE::G, LZ = GE::LZ, LP = GE::LP, KZP = GE::KZP;
    constexpr bool Z3 = (N % 3 == 0) && (PS_Z3 != 0);
    constexpr int M = Z3 ? N / 3 : N;
    constexpr int GM = LineFFT<T, M, 1>::G;        // threads per sub-line
    static_assert(!Z3 || G == 3 * GM, "three sub-lines per line group");
    // a (sub-)line's threads are consecutive and start at a multiple of its
    // thread count: if that count divides 32, its stages need warp barriers only
    constexpr int GL = Z3 ? GM : G;
    constexpr bool WS = PS_ZWS != 0 && GL <= 32 && 32 % GL == 0;
    constexpr int TWM = Z3 ? (tw_count(M) > 0 ? tw_count(M) : 1) : 0;
    constexpr int nyl = NY;   // lines per x-plane (= kp.n; the line length is N)
    const int b0 = kp.xs0 * nyl / LZ, b1 = (kp.xs0 + kp.xsn) * nyl / LZ;   // this launch's batches
    constexpr uint32_t fbytes = (uint32_t)(LZ * KZP * sizeof(C2));
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int NB = GE::ZNB;
    C2* stage = reinterpret_cast<C2*>(smem_base128(smraw));   // [NB][6][LZ][KZP]
    if (smem_u32(stage) & 127u) {   // never expected: refuse to start copies
        if (threadIdx.x == 0) atomicExch(err, 2);
        return;
    }
    C2* tiles = stage + NB * 6 * LZ * KZP;               // [LZ][3][LP]
    C2* tw = tiles + 3 * LZ * LP;
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ double wacc[32][12];     // per-warp (sum, compensation) of the six sums
    __shared__ uint8_t sflag[LZ];       // mask flags of the batch's lines
    const int fl = threadIdx.x / G, g = threadIdx.x % G;
    const int pl = fl / 3, pr = fl % 3;
    const int Kz = kp.Kz;
    const size_t BS = (size_t)nyl * nyl * KZP;
    auto tile = [&](int l, int p) { return tiles + (size_t)(l * 3 + p) * LP; };
    auto zad = [](int p) { return p + (p >> 4); };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    C2* tw3 = tw + TWM;   // n = 3M: e^{+2 pi i b q'/n}, b = 1, 2
    if constexpr (Z3) {
        if constexpr (tw_count(M) > 0) load_tw(tw, twg + N, tw_count(M));
        load_tw(tw3, twg + 2 * N, 2 * M);
    } else {
        load_tw(tw, twg, GE::tw_n);
    }
    for (int i = threadIdx.x; i < 32 * 12; i += blockDim.x) (&wacc[0][0])[i] = 0.0;
    __syncthreads();
    auto issue = [&](int b, int buf) {  // one thread
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar[buf], 6 * fbytes);
        // kept rolled: fully unrolled, the six copies crashed ptxas 13.0 at n = 768
#pragma unroll 1
        for (int f = 0; f < 6; ++f)
            bulk_g2s(stage + (size_t)(buf * 6 + f) * LZ * KZP, B + f * BS + (size_t)b * LZ * KZP, fbytes, &bar[buf]);
    };
    if (threadIdx.x == 0 && b0 + (int)blockIdx.x < b1) issue(b0 + blockIdx.x, 0);

    const size_t N3 = (size_t)nyl * nyl * N;
    const T inv_eta = (T)kp.inv_eta;
    int it = 0;
    for (int b = b0 + blockIdx.x; b < b1; b += gridDim.x, ++it) {
        const int buf = NB == 2 ? (it & 1) : 0;
        const bool more = b + (int)gridDim.x < b1;
        if (NB == 2 && threadIdx.x == 0 && more) issue(b + gridDim.x, buf ^ 1);
        const uint32_t par = NB == 2 ? (uint32_t)((it >> 1) & 1) : (uint32_t)(it & 1);
        const bool ok = mbar_wait(&bar[buf], par);
        if (__syncthreads_or(!ok)) {
            // a copy never completed: record it, let any copy in flight land, stop
            if (threadIdx.x == 0) {
                atomicExch(err, 1);
                if (NB == 1) mbar_wait(&bar[0], par);
                else if (more) mbar_wait(&bar[buf ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
            }
            break;
        }
        const C2* st = stage + (size_t)buf * 6 * LZ * KZP;
        // the batch's mask flags: loaded now, stored to shared memory after
        // the inverse transforms, read by the pointwise phase
        const uint8_t myflag = threadIdx.x < LZ ? flag[(size_t)b * LZ + threadIdx.x] : (uint8_t)0;
        if constexpr (Z3) {
            // the split's pre-butterfly once per mirror pair of modes, into the
            // tiles; each thread group fills its own tile (pl, pr)
            {
                const C2* fa = st + (size_t)((2 * pr) * LZ + pl) * KZP;
                const C2* fb = st + (size_t)((2 * pr + 1) * LZ + pl) * KZP;
                C2* t = tile(pl, pr);
                for (int q = g; q < M / 2; q += G) split3_pre<T, M>(fa, fb, tw3, t, q);
            }
            __syncthreads();
            // one buffer: every read of it is done, the next batch may land
            if (NB == 1 && threadIdx.x == 0 && more) issue(b + gridDim.x, 0);
            const int sub = g / GM, gm = g % GM;
            const int tbase = (int)(tile(pl, pr) - tiles);
            auto noload = [&](int) -> C2 { return cmk<C2>((T)0, (T)0); };
            if constexpr (M % 16 == 0) {   // the sub-line starts on a padding group
                LineFFT<T, M, 1, WS>::template run_tile<true>(tiles, tw, Pad16{tbase + zad(sub * M)}, gm, noload);
            } else {
                auto addr = [&](int p) { return tbase + zad(sub * M + p); };
                auto store = [&](int p, C2 v) { tiles[addr(p)] = v; };
                LineFFT<T, M, 1, WS>::template run<true>(tiles, tw, addr, gm, noload, store);
            }
        } else {
            const C2* fa = st + (size_t)((2 * pr) * LZ + pl) * KZP;
            const C2* fb = st + (size_t)((2 * pr + 1) * LZ + pl) * KZP;
            const int tbase = (int)(tile(pl, pr) - tiles);
            auto load = [&](int q) -> C2 {
                if (q < Kz) {
                    C2 a = fa[q], c = fb[q];
                    if (q == 0) { a.y = 0; c.y = 0; }
                    return cmk<C2>(a.x - c.y, a.y + c.x);          // A + i B
                }
                if (q > N - Kz) {
                    const C2 a = fa[N - q], c = fb[N - q];
                    return cmk<C2>(a.x + c.y, c.x - a.y);          // conj(A) + i conj(B)
                }
                return cmk<C2>((T)0, (T)0);
            };
            LineFFT<T, N, 1, WS>::template run_tile<false>(tiles, tw, Pad16{tbase}, g, load);
        }
        if (threadIdx.x < LZ) sflag[threadIdx.x] = myflag;
        __syncthreads();
        // one buffer: every read of it is done, the next batch may land
        if (!Z3 && NB == 1 && threadIdx.x == 0 && more) issue(b + gridDim.x, 0);
        double fm[6] = {0, 0, 0, 0, 0, 0};
        bool touched = false;
        // n = u x w - (chi/eta)(u - us) of line l at z; forces in double
        auto nonlinear = [&](int l, int z, int a, T& nx, T& ny, T& nz) {
            const long lid = (long)b * LZ + l;
            const C2 z0 = tile(l, 0)[a], z1 = tile(l, 1)[a], z2 = tile(l, 2)[a];
            const T ux = z0.x, uy = z0.y, uz = z1.x, wx = z1.y, wy = z2.x, wz = z2.y;
            nx = uy * wz - uz * wy;
            ny = uz * wx - ux * wz;
            nz = ux * wy - uy * wx;
            if constexpr (PM) half_u2[(size_t)lid * N + z] = (T)0.5 * (ux * ux + uy * uy + uz * uz);
            if (sflag[l] != 0) {
                const size_t po = (size_t)lid * N + z;
                const T c = chi[po];
                if (c != (T)0) {
                    const int x = (int)(lid / nyl), y = (int)(lid % nyl);
                    const T sx = us[po], sy = us[N3 + po], sz = us[2 * N3 + po];
                    const T ce = c * inv_eta;
                    nx -= ce * (ux - sx);
                    ny -= ce * (uy - sy);
                    nz -= ce * (uz - sz);
                    const double cd = (double)c;
                    const double px = cd * ((double)ux - (double)sx);
                    const double py = cd * ((double)uy - (double)sy);
                    const double pz = cd * ((double)uz - (double)sz);
                    const double rx = x * kp.dx - kp.x0[0], ry = y * kp.dx - kp.x0[1], rz = z * kp.dx - kp.x0[2];
                    fm[0] += px;
                    fm[1] += py;
                    fm[2] += pz;
                    fm[3] += ry * pz - rz * py;
                    fm[4] += rz * px - rx * pz;
                    fm[5] += rx * py - ry * px;
                    touched = true;
                }
            }
        };
        // lines 2m and 2m+1 together: (n_x + i n_y) of each in place of
        // (u_x + i u_y), and (n_z[2m] + i n_z[2m+1]) in place of line 2m's
        // (u_z + i w_x); this thread alone reads and writes these slots
        for (int idx = threadIdx.x; idx < (LZ / 2) * N; idx += blockDim.x) {
            const int l = 2 * (idx / N), r = idx % N;
            // tile position r holds z = r (n = 3M: z = 3 (r mod M) + r / M)
            const int z = Z3 ? 3 * (r % M) + r / M : r;
            const int a = zad(r);
            T nx0, ny0, nz0, nx1, ny1, nz1;
            nonlinear(l, z, a, nx0, ny0, nz0);
            nonlinear(l + 1, z, a, nx1, ny1, nz1);
            if constexpr (SP) {
                // s = chi_sp omega of both lines, read before their slots are reused
                const long lid0 = (long)b * LZ + l;
                const T c0 = chi_sp[(size_t)lid0 * N + z], c1 = chi_sp[(size_t)(lid0 + 1) * N + z];
                const T wx0 = tile(l, 1)[a].y, wx1 = tile(l + 1, 1)[a].y;
                const C2 w0 = tile(l, 2)[a], w1 = tile(l + 1, 2)[a];
                tile(l, 2)[a] = cmk<C2>(c0 * wx0, c0 * w0.x);
                tile(l + 1, 2)[a] = cmk<C2>(c1 * wx1, c1 * w1.x);
                tile(l + 1, 1)[a] = cmk<C2>(c0 * w0.y, c1 * w1.y);
            }
            tile(l, 0)[a] = cmk<C2>(nx0, ny0);
            tile(l + 1, 0)[a] = cmk<C2>(nx1, ny1);
            tile(l, 1)[a] = cmk<C2>(nz0, nz1);
        }
        // this batch's force sums: warp tree, then compensated into the warp slot
        if (__any_sync(0xffffffffu, touched)) {
            for (int i = 0; i < 6; ++i)
                for (int o = 16; o > 0; o >>= 1) fm[i] += __shfl_down_sync(0xffffffffu, fm[i], o);
            if ((threadIdx.x & 31) == 0) {
                double* w = wacc[threadIdx.x >> 5];
                for (int i = 0; i < 6; ++i) {
                    Acc a = {w[2 * i], w[2 * i + 1]};
                    a.add(fm[i]);
                    w[2 * i] = a.s;
                    w[2 * i + 1] = a.c;
                }
            }
        }
        __syncthreads();
        {
            // forward lines: (l, 0) for every l, (l, 1) for even l; others idle
            // (with the sponge: every tile)
            const bool active = SP || (pr == 0) || (pr == 1 && (pl & 1) == 0);
            const int tbase = (int)(tile(pl, SP ? pr : (pr == 2 ? 1 : pr)) - tiles);
            auto noload = [&](int) -> C2 { return cmk<C2>((T)0, (T)0); };
            if constexpr (Z3) {
                const int sub = g / GM, gm = g % GM;
                if constexpr (M % 16 == 0) {
                    LineFFT<T, M, -1, WS>::template run_tile_masked<true>(tiles, tw, Pad16{tbase + zad(sub * M)}, gm,
                                                                          noload, active);
                } else {
                    auto addr = [&](int p) { return tbase + zad(sub * M + p); };
                    auto store = [&](int p, C2 v) { if (active) tiles[addr(p)] = v; };
                    LineFFT<T, M, -1, WS>::template run_masked<true>(tiles, tw, addr, gm, noload, store, active);
                }
            } else {
                LineFFT<T, N, -1, WS>::template run_tile_masked<true>(tiles, tw, Pad16{tbase}, g, noload, active);
            }
        }
        __syncthreads();
        C2* const Bw = PM ? Bo : B;
        // P = (Z_k + conj Z_{-k}) / 2 and Q = (Z_k - conj Z_{-k}) / (2 i) of a two-for-one transform
        auto P2 = [](C2 zk, C2 zm) { return cmk<C2>((T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y)); };
        auto Q2 = [](C2 zk, C2 zm) { return cmk<C2>((T)0.5 * (zk.y + zm.y), (T)0.5 * (zm.x - zk.x)); };
        if constexpr (Z3) {
            // radix-3 recombination of the sub-line spectra by mirror pairs of
            // kept modes, unpacked straight to B: tile (l, 0) -> fields 0, 1 of
            // line l; (l, 1), l even -> field 2 of lines l, l + 1; with the
            // sponge also (l, 2) -> fields 3, 4 of line l and (l, 1), l odd ->
            // field 5 of lines l - 1, l
            constexpr int NT = SP ? 3 * LZ : LZ + LZ / 2;   // transformed tiles
            for (int idx = threadIdx.x; idx < NT * (M / 2); idx += blockDim.x) {
                const int tj = idx / (M / 2), k = idx % (M / 2);
                const int l = SP ? tj % LZ : (tj < LZ ? tj : 2 * (tj - LZ));
                const int p = SP ? tj / LZ : (tj < LZ ? 0 : 1);
                const size_t lo = ((size_t)b * LZ + l) * KZP;
                C2 *dP, *dQ;
                if (p == 0) {
                    dP = Bw + lo;
                    dQ = Bw + BS + lo;
                } else if (p == 2) {
                    dP = B + 3 * BS + lo;
                    dQ = B + 4 * BS + lo;
                } else if ((l & 1) == 0) {
                    dP = Bw + 2 * BS + lo;
                    dQ = Bw + 2 * BS + lo + KZP;
                } else {
                    dP = B + 5 * BS + lo - KZP;
                    dQ = B + 5 * BS + lo;
                }
                C2 zk, znk, zm, znm;
                split3_pair_out<T, M>(tile(l, p), tw3, k, zk, znk, zm, znm);
                const int k2 = k == 0 ? M / 2 : M - k;
                dP[k] = P2(zk, znk);
                dQ[k] = Q2(zk, znk);
                dP[k2] = P2(zm, znm);
                dQ[k2] = Q2(zm, znm);
            }
        } else {
            // unpack the two-for-one transforms, keep kz < Kz
            for (int idx = threadIdx.x; idx < LZ * Kz; idx += blockDim.x) {
                const int l = idx / Kz, k = idx % Kz;
                const size_t lo = ((size_t)b * LZ + l) * KZP;
                const C2* t0 = tile(l, 0);
                const C2* t1 = tile(l & ~1, 1);
                const int m = (N - k) % N;
                const C2 zk = t0[zad(k)], zm = t0[zad(m)];
                Bw[lo + k] = P2(zk, zm);
                Bw[BS + lo + k] = Q2(zk, zm);
                const C2 wk = t1[zad(k)], wm = t1[zad(m)];
                Bw[2 * BS + lo + k] = (l & 1) ? Q2(wk, wm) : P2(wk, wm);
                if constexpr (SP) {
                    const C2* t2 = tile(l, 2);
                    const C2* t3 = tile(l | 1, 1);
                    const C2 sk = t2[zad(k)], sm = t2[zad(m)];
                    B[3 * BS + lo + k] = P2(sk, sm);
                    B[4 * BS + lo + k] = Q2(sk, sm);
                    const C2 qk = t3[zad(k)], qm = t3[zad(m)];
                    B[5 * BS + lo + k] = (l & 1) ? Q2(qk, qm) : P2(qk, qm);
                }
            }
        }
        __syncthreads();
    }
    __syncthreads();
    if (!PM && threadIdx.x < 6) {
        Acc a = {0, 0};
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) {
            a.add(wacc[w][2 * threadIdx.x]);
            a.add(wacc[w][2 * threadIdx.x + 1]);
        }
        partial[(size_t)(kp.part_off + blockIdx.x) * 6 + threadIdx.x] = a.val();
    }
}

// ---------------------------------------------------------------- pass 4
template <typename T, int N>
__global__ void __launch_bounds__(Geo<T, N>::C * Geo<T, N>::G)
k_yfwd(KP kp, const cplx<T>* __restrict__ B, cplx<T>* __restrict__ A, const cplx<T>* __restrict__ twg) {
    using C2 = cplx<T>;
    using GE = Geo<T, N>;
    constexpr int C = GE::C;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* tw = reinterpret_cast<C2*>(smraw);
    C2* tile = tw + GE::tw_n;
    const int col = threadIdx.x % C, g = threadIdx.x / C;
    const int cz = blockIdx.x * C + col;
    const bool okz = cz < kp.Kz;
    const int x = blockIdx.y;
    const int K = kp.K, mmax = kp.mmax, Kzp = kp.Kzp;
    const size_t AS = (size_t)N * K * Kzp;
    const size_t BS = (size_t)N * N * Kzp;
    load_tw(tw, twg, GE::tw_n);
    auto addr = [&](int p) { return p * C + col; };
#pragma unroll 1
    for (int f = 0; f < 3; ++f) {
        __syncthreads();
        auto load = [&](int y) -> C2 {
            if (!okz) return cmk<C2>((T)0, (T)0);
            return B[f * BS + ((size_t)x * N + y) * Kzp + cz];
        };
        auto store = [&](int q, C2 v) {
            const int m = mode_of(q, N);
            if (okz && m <= mmax && m >= -mmax) A[f * AS + GE::arow(x, cidx_of(m, K)) * Kzp + cz] = v;
        };
        LineFFT<T, N, -1>::template run<false>(tile, tw, addr, g, load, store);
    }
}

// ---------------------------------------------------------------- pass 5
// MODE 0: time step (Euler if first != 0, else AB2); MODE 1: set velocity
// (project with the mean kept, history cleared); MODE 2: plain truncated
// forward transform (times 1/n^3) into U, H untouched.
template <typename T, int N, int MODE>
__global__ void __launch_bounds__(Geo<T, N>::C5 * Geo<T, N>::G)
k_xfwd(KP kp, const cplx<T>* __restrict__ A, cplx<T>* __restrict__ U, cplx<T>* __restrict__ H,
       const T* __restrict__ Ex, const T* __restrict__ Ez, int first, const cplx<T>* __restrict__ twg) {
    using C2 = cplx<T>;
    using GE = Geo<T, N>;
    constexpr int C = GE::C5;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* tw = reinterpret_cast<C2*>(smraw);
    C2* tiles = tw + GE::tw_n;
    const int col = threadIdx.x % C, g = threadIdx.x / C;
    const int cz0 = blockIdx.x * C;
    const int cz = cz0 + col;
    const bool okz = cz < kp.Kz;
    const int cy = blockIdx.y;
    const int K = kp.K, mmax = kp.mmax, Kzp = kp.Kzp;
    const size_t AS = (size_t)N * K * Kzp;
    const size_t FS = (size_t)K * K * Kzp;
    load_tw(tw, twg, GE::tw_n);
    auto addr = [&](int p) { return p * C + col; };
#pragma unroll 1
    for (int f = 0; f < 3; ++f) {
        C2* tile = tiles + f * N * C;
        __syncthreads();
        auto load = [&](int x) -> C2 {
            if (!okz) return cmk<C2>((T)0, (T)0);
            return A[f * AS + GE::arow(x, cy) * Kzp + cz];
        };
        auto store = [&](int q, C2 v) { tile[addr(q)] = v; };
        LineFFT<T, N, -1>::template run<false>(tile, tw, addr, g, load, store);
    }
    __syncthreads();
    const T s = (T)kp.ks, sz = (T)kp.ksz;
    const T my = (T)cmode_of(cy, mmax, K);
    const T invn3 = (T)kp.invn3;
    const T dt = (T)kp.dt;
    const T ey = Ex[cy];
    for (int idx = threadIdx.x; idx < K * C; idx += blockDim.x) {
        const int cx = idx / C, c = idx % C;
        const int czz = cz0 + c;
        if (czz >= kp.Kz) continue;
        const int mx = cmode_of(cx, mmax, K);
        const int q = mx >= 0 ? mx : mx + N;
        const int a = q * C + c;
        C2 n0 = tiles[a], n1 = tiles[N * C + a], n2 = tiles[2 * N * C + a];
        n0.x *= invn3; n0.y *= invn3;
        n1.x *= invn3; n1.y *= invn3;
        n2.x *= invn3; n2.y *= invn3;
        const T kx = s * (T)mx, ky = s * my, kz = sz * (T)czz;
        const T k2 = kx * kx + ky * ky + kz * kz;
        const bool zero = (mx == 0 && cy == 0 && czz == 0);
        const size_t o = ((size_t)cy * K + cx) * Kzp + czz;
        if constexpr (MODE == 2) {   // plain truncated forward transform into U
            U[o] = n0; U[FS + o] = n1; U[2 * FS + o] = n2;
            continue;
        }
        if (!zero) {
            const T ik2 = (T)1 / k2;
            const T dr = (kx * n0.x + ky * n1.x + kz * n2.x) * ik2;
            const T di = (kx * n0.y + ky * n1.y + kz * n2.y) * ik2;
            n0.x -= kx * dr; n0.y -= kx * di;
            n1.x -= ky * dr; n1.y -= ky * di;
            n2.x -= kz * dr; n2.y -= kz * di;
        } else if (MODE == 0 && !kp.mean_free) {
            n0 = n1 = n2 = cmk<C2>((T)0, (T)0);
        }
        if constexpr (MODE == 1) {
            U[o] = n0; U[FS + o] = n1; U[2 * FS + o] = n2;
            const C2 z = cmk<C2>((T)0, (T)0);
            H[o] = z; H[FS + o] = z; H[2 * FS + o] = z;
        } else {
            const T E = Ex[cx] * ey * Ez[czz];
            C2 nn[3] = {n0, n1, n2};
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const C2 uq = first ? U[f * FS + o] : H[f * FS + o];
                C2 un, qn;
                ab2_update(uq, nn[f], E, dt, first != 0, un, qn);
                U[f * FS + o] = un;
                H[f * FS + o] = qn;
            }
        }
    }
}

// --------------------------------------------- TMA-staged y passes
// Persistent blocks walk a list of items (x plane, kz tile of CT columns,
// field); each item's input tile arrives by tiled TMA copies into one of two
// staging buffers while the previous item is transformed.

// pass 2: y-inverse of the NF (6, or 3 for a plain 3-field transform)
// fields, A (kept ky rows) -> B (all y rows); one staging buffer, refilled
// once the first FFT stage has read it.
// tm: A as {2 Kzp reals, n rows (x), 6 K planes (f K + ky)}.
// KZP_: kz columns of the spectral arrays (compile time: the address
// arithmetic folds into immediate offsets; the n x n x n/2 engines pass the
// value of their z length).
template <typename T, int N, int NF = 6, int KZP_ = Geo<T, N>::KZP>
__global__ void __launch_bounds__(Geo<T, N>::CY2 * Geo<T, N>::G)
k_yinv_tma(const __grid_constant__ CUtensorMap tm, KP kp, cplx<T>* __restrict__ B, const cplx<T>* __restrict__ twg,
           int* __restrict__ err) {
    using C2 = cplx<T>;
    using GE = Geo<T, N>;
    constexpr int CT = GE::CY2, G = GE::G, K = GE::K;
    constexpr int NBOX = GE::nbox(K), BR = GE::brows(K), BP = GE::bpitch(K, CT), RS = NBOX * BP;
    constexpr int KZP = KZP_, NTZ = KZP / CT;
    const int NITEM = kp.xsn * NTZ * NF;  // items of this launch's x planes
    constexpr uint32_t box_bytes = (uint32_t)(BR * CT * sizeof(C2));
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int NB = GE::Y2NB;
    C2* S = reinterpret_cast<C2*>(smem_base128(smraw));   // [NB][RS][CT]
    if (smem_u32(S) & 127u) {   // never expected: refuse to start copies
        if (threadIdx.x == 0) atomicExch(err, 2);
        return;
    }
    C2* W = S + NB * RS * CT;                             // [N][CT]
    C2* tw = W + N * CT;
    __shared__ __align__(8) uint64_t bar[2];
    const int col = threadIdx.x % CT, g = threadIdx.x / CT;
    const int mmax = kp.mmax, Kz = kp.Kz;
    const size_t BS = (size_t)N * N * KZP;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    load_tw(tw, twg, GE::tw_n);
    __syncthreads();
    auto issue = [&](int i, int buf) {  // one thread
        const int f = i % NF, t = i / NF, x = kp.xs0 + t / NTZ, czt = t % NTZ;
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar[buf], NBOX * box_bytes);
        for (int b = 0; b < NBOX; ++b)
            tma_load_3d(S + (size_t)(buf * RS + b * BP) * CT, &tm, 2 * czt * CT, x, f * K + b * BR, &bar[buf]);
    };
    if (threadIdx.x == 0 && (int)blockIdx.x < NITEM) issue(blockIdx.x, 0);
    auto addr = [&](int p) { return p * CT + col; };
    int it = 0;
    using FFT = LineFFT<T, N, 1>;
    for (int i = blockIdx.x; i < NITEM; i += gridDim.x, ++it) {
        const int buf = NB == 2 ? (it & 1) : 0;
        const bool more = i + (int)gridDim.x < NITEM;
        if (NB == 2 && threadIdx.x == 0 && more) issue(i + gridDim.x, buf ^ 1);
        const uint32_t par = NB == 2 ? (uint32_t)((it >> 1) & 1) : (uint32_t)(it & 1);
        const bool ok = mbar_wait(&bar[buf], par);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicExch(err, 1);
                if (NB == 1) mbar_wait(&bar[0], par);
                else if (more) mbar_wait(&bar[buf ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
            }
            break;
        }
        const int f = i % NF, t = i / NF, x = kp.xs0 + t / NTZ, czt = t % NTZ;
        const int cz = czt * CT + col;
        const bool okz = cz < Kz;
        const C2* Sb = S + (size_t)buf * RS * CT;
        auto load = [&](int q) -> C2 {
            const int m = mode_of(q, N);
            if (m > mmax || m < -mmax) return cmk<C2>((T)0, (T)0);
            const int c = cidx_of(m, K);
            return Sb[((c / BR) * BP + c % BR) * CT + col];
        };
        auto store = [&](int y, C2 v) {
            if (okz) B[f * BS + ((size_t)x * N + y) * KZP + cz] = v;
        };
        if constexpr (NB == 1 && FFT::S > 1) {
            // one buffer: refill it once the first stage has read it
            auto refill = [&]() {
                if (threadIdx.x == 0 && more) issue(i + gridDim.x, 0);
            };
            FFT::template run_hook<false>(W, tw, addr, g, load, store, refill);
            __syncthreads();
        } else {
            FFT::template run<false>(W, tw, addr, g, load, store);
            __syncthreads();
            if (NB == 1 && threadIdx.x == 0 && more) issue(i + gridDim.x, 0);
        }
    }
}

// pass 4: y-forward of the three fields, B (all y rows) -> A (kept ky rows).
// tm: B as a 2-D array of 6 n n rows of 2 Kzp reals.
template <typename T, int N, int CTV, int NF = 3, int KZP_ = Geo<T, N>::KZP>
__global__ void __launch_bounds__(CTV * Geo<T, N>::G)
k_yfwd_tma(const __grid_constant__ CUtensorMap tm, KP kp, cplx<T>* __restrict__ A, const cplx<T>* __restrict__ twg,
           int* __restrict__ err) {
    using C2 = cplx<T>;
    using GE = Geo<T, N>;
    constexpr int CT = CTV, G = GE::G, K = GE::K;
    constexpr int NBOX = GE::nbox(N), BR = GE::brows(N), BP = GE::bpitch(N, CT), RS = NBOX * BP;
    static_assert(NBOX == 1 || BR == BP, "y-forward staging must be contiguous in y");
    constexpr int KZP = KZP_, NTZ = KZP / CT;
    const int NITEM = kp.xsn * NTZ * NF;   // items of this launch's x planes
    constexpr uint32_t box_bytes = (uint32_t)(BR * CT * sizeof(C2));
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* S = reinterpret_cast<C2*>(smem_base128(smraw));   // [2][RS][CT]
    if (smem_u32(S) & 127u) {   // never expected: refuse to start copies
        if (threadIdx.x == 0) atomicExch(err, 2);
        return;
    }
    C2* tw = S + 2 * RS * CT;
    __shared__ __align__(8) uint64_t bar[2];
    const int col = threadIdx.x % CT, g = threadIdx.x / CT;
    const int mmax = kp.mmax, Kz = kp.Kz;
    const size_t AS = (size_t)N * K * KZP;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    using S3 = Split3<T, N>;
    const C2* tw3 = load_tw_split<T, N>(tw, twg, GE::tw_n);
    __syncthreads();
    auto issue = [&](int i, int buf) {  // one thread
        const int f = i % NF, t = i / NF, x = kp.xs0 + t / NTZ, czt = t % NTZ;
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar[buf], NBOX * box_bytes);
        for (int b = 0; b < NBOX; ++b)
            tma_load_2d(S + (size_t)(buf * RS + b * BP) * CT, &tm, 2 * czt * CT, (f * N + x) * N + b * BR, &bar[buf]);
    };
    if (threadIdx.x == 0 && (int)blockIdx.x < NITEM) issue(blockIdx.x, 0);
    int it = 0;
    for (int i = blockIdx.x; i < NITEM; i += gridDim.x, ++it) {
        const int buf = it & 1;
        const bool more = i + (int)gridDim.x < NITEM;
        if (threadIdx.x == 0 && more) issue(i + gridDim.x, buf ^ 1);
        const bool ok = mbar_wait(&bar[buf], (uint32_t)((it >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicExch(err, 1);
                if (more) mbar_wait(&bar[buf ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
            }
            break;
        }
        const int f = i % NF, t = i / NF, x = kp.xs0 + t / NTZ, czt = t % NTZ;
        const int cz = czt * CT + col;
        const bool okz = cz < Kz;
        C2* Sb = S + (size_t)buf * RS * CT;
        auto noload = [&](int) -> C2 { return cmk<C2>((T)0, (T)0); };
        if constexpr (S3::on) {
            // sub-line b = rows y = 3a + b, transformed in place; then the
            // kept outputs by the radix-3 recombination
            constexpr int M = S3::M;
            const int sub = g / S3::GM, gm = g % S3::GM;
            auto addr3 = [&](int p) { return (int)(Sb - S) + (3 * p + sub) * CT + col; };
            auto store = [&](int p, C2 v) { S[addr3(p)] = v; };
            LineFFT<T, M, -1>::template run<true>(S, tw, addr3, gm, noload, store);
            __syncthreads();
            for (int idx = threadIdx.x; idx < M * CT; idx += blockDim.x) {
                const int kq = idx / CT, c = idx % CT;
                const int czz = czt * CT + c;
                C2 Zk, Zm;
                split3_out(Sb[(3 * kq) * CT + c], Sb[(3 * kq + 1) * CT + c], Sb[(3 * kq + 2) * CT + c], tw3, kq, M,
                           Zk, Zm);
                if (czz < Kz) {
                    C2* o = A + f * AS + czz;
                    o[GE::arow(x, kq) * KZP] = Zk;                             // mode kq
                    if (kq > 0) o[GE::arow(x, kq + M - 1) * KZP] = Zm;         // mode kq - M
                }
            }
        } else {
            auto addr = [&](int p) { return (int)(Sb - S) + p * CT + col; };
            auto store = [&](int q, C2 v) {
                const int m = mode_of(q, N);
                if (okz && m <= mmax && m >= -mmax) A[f * AS + GE::arow(x, cidx_of(m, K)) * KZP + cz] = v;
            };
            LineFFT<T, N, -1>::template run<true>(S, tw, addr, g, noload, store);
        }
        __syncthreads();
    }
}

// pass 1 (TMA-staged): x-inverse of u and omega = curl u with five
// transforms per (cy, kz tile): Ux, Uy, Dx Uy = F[i kx u_y], Uz, Dx Uz.
// Along an x line ky and kz are constant, so after the x transform
//   w_x = i (ky Uz - kz Uy),  w_y = i kz Ux - Dx Uz,  w_z = Dx Uy - i ky Ux;
// a thread keeps its last-stage outputs of Ux and Uy in registers until the
// transforms that need them. Inputs arrive field by field (x, y, z) by TMA.
// NF = 3: the plain x-inverse of three fields (one transform each, no curl).
// tm: U (or the array being transformed) as 2-D rows of 2 Kzp reals, row
// (f K + cy) K + cx.
template <typename T, int N, int NF = 6, int KZP_ = Geo<T, N>::KZP>
__global__ void __launch_bounds__(Geo<T, N>::CX1 * Geo<T, N>::G)
k_xinv_tma(const __grid_constant__ CUtensorMap tm, KP kp, cplx<T>* __restrict__ A, const cplx<T>* __restrict__ twg,
           int* __restrict__ err) {
    using C2 = cplx<T>;
    using GE = Geo<T, N>;
    using FFT = LineFFT<T, N, 1>;
    constexpr int CT = GE::CX1, G = GE::G, K = GE::K;
    constexpr int NBOX = GE::nbox(K), BR = GE::brows(K), BP = GE::bpitch(K, CT), RS = NBOX * BP;
    constexpr int KZP = KZP_, NTZ = KZP / CT;
    const int NTILE = kp.kyn * NTZ;   // tiles of this launch's ky rows
    constexpr uint32_t box_bytes = (uint32_t)(BR * CT * sizeof(C2));
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* S = reinterpret_cast<C2*>(smem_base128(smraw));   // [2][RS][CT]
    if (smem_u32(S) & 127u) {
        if (threadIdx.x == 0) atomicExch(err, 2);
        return;
    }
    C2* W = S + 2 * RS * CT;                              // [N][CT]
    C2* tw = W + N * CT;
    __shared__ __align__(8) uint64_t bar[2];
    const int col = threadIdx.x % CT, g = threadIdx.x / CT;
    const int mmax = kp.mmax, Kz = kp.Kz;
    const T ks = (T)kp.ks, ksz = (T)kp.ksz;   // wavenumbers in T: no double arithmetic per element
    const size_t AS = (size_t)N * K * KZP;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    load_tw(tw, twg, GE::tw_n);
    __syncthreads();
    // load L: tile iteration L / 3, field L % 3
    auto issue = [&](int L) {  // one thread
        const int t = blockIdx.x + (L / 3) * gridDim.x, f = L % 3, buf = L & 1;
        if (t >= NTILE) return;
        const int cy = kp.ky0 + t / NTZ, czt = t % NTZ;
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar[buf], NBOX * box_bytes);
        for (int b = 0; b < NBOX; ++b)
            tma_load_2d(S + (size_t)(buf * RS + b * BP) * CT, &tm, 2 * czt * CT, (f * K + cy) * K + b * BR, &bar[buf]);
    };
    if (threadIdx.x == 0) issue(0);
    auto addr = [&](int p) { return p * CT + col; };
    C2 R1[FFT::SLOTS], R2[FFT::SLOTS];
    int ti = 0;
    bool stop = false;
    for (int t = blockIdx.x; t < NTILE && !stop; t += gridDim.x, ++ti) {
        const int cy = kp.ky0 + t / NTZ, czt = t % NTZ;
        const int cz = czt * CT + col;
        const bool okz = cz < Kz;
        const T ky = ks * (T)cmode_of(cy, mmax, K);
        const T kz = ksz * (T)cz;
        C2* out = A + cz;   // + f AS + arow(x, cy) KZP
#pragma unroll 1
        for (int f = 0; f < 3; ++f) {
            const int L = 3 * ti + f, buf = L & 1;
            if (threadIdx.x == 0) issue(L + 1);
            const bool ok = mbar_wait(&bar[buf], (uint32_t)((L >> 1) & 1));
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) {
                    atomicExch(err, 1);
                    mbar_wait(&bar[buf ^ 1], (uint32_t)(((L + 1) >> 1) & 1));
                }
                stop = true;
                break;
            }
            const C2* Sb = S + (size_t)buf * RS * CT;
#pragma unroll 1
            for (int d = 0; d < (NF == 6 && f > 0 ? 2 : 1); ++d) {
                // d = 1: the x derivative i kx u_f
                auto load = [&](int q) -> C2 {
                    const int m = mode_of(q, N);
                    if (m > mmax || m < -mmax) return cmk<C2>((T)0, (T)0);
                    const int c = cidx_of(m, K);
                    const C2 v = Sb[((c / BR) * BP + c % BR) * CT + col];
                    if (d == 0) return v;
                    const T kx = ks * (T)m;
                    return cmk<C2>(-kx * v.y, kx * v.x);
                };
                auto store = [&](int slot, int x, C2 v) {
                    C2* o = out + GE::arow(x, cy) * KZP;
                    if constexpr (NF == 3) {            // plain: field f only
                        if (okz) o[f * AS] = v;
                        return;
                    }
                    if (f == 0) {                       // Ux
                        R1[slot] = v;
                        if (okz) o[0] = v;
                    } else if (f == 1 && d == 0) {      // Uy
                        R2[slot] = v;
                        if (okz) o[AS] = v;
                    } else if (f == 1) {                // w_z = Dx Uy - i ky Ux
                        const C2 u = R1[slot];
                        if (okz) o[5 * AS] = cmk<C2>(v.x + ky * u.y, v.y - ky * u.x);
                    } else if (d == 0) {                // Uz; w_x = i (ky Uz - kz Uy)
                        const C2 u = R2[slot];
                        if (okz) {
                            o[2 * AS] = v;
                            o[3 * AS] = cmk<C2>(-(ky * v.y - kz * u.y), ky * v.x - kz * u.x);
                        }
                    } else {                            // w_y = i kz Ux - Dx Uz
                        const C2 u = R1[slot];
                        if (okz) o[4 * AS] = cmk<C2>(-kz * u.y - v.x, kz * u.x - v.y);
                    }
                };
                FFT::template run_bu<false>(W, tw, addr, g, load, store);
                __syncthreads();
            }
        }
    }
}

// pass 5 (TMA-staged): x-forward of the three fields of n, truncation to the
// kept kx, 1/n^3, Leray projection and the integrating-factor AB2 (Euler on
// the first step) update of U and H. MODE 1 instead sets U to the projected
// field (mean kept) and clears H; MODE 2 writes the truncated transform
// times 1/n^3 to U (no projection; H unused); MODE 3 writes the total
// pressure coefficients Pi_hat = -i (k . N_hat) / |k|^2 (one field) to U,
// the gradient part the projection removes. Each field is transformed in
// place in its staging buffer; kept outputs go to three result tiles.
// tm: A as rows of 2 Kzp reals, row (f K + ky) n + x.
template <typename T, int N, int MODE, bool SP = false, int KZP_ = Geo<T, N>::KZP>
__global__ void __launch_bounds__(Geo<T, N>::CX5 * Geo<T, N>::G)
k_xfwd_tma(const __grid_constant__ CUtensorMap tm, const __grid_constant__ CUtensorMap tmu,
           const __grid_constant__ CUtensorMap tmh, KP kp, cplx<T>* __restrict__ U, cplx<T>* __restrict__ H,
           const T* __restrict__ Ex, const T* __restrict__ Ez, int first, const cplx<T>* __restrict__ twg,
           int* __restrict__ err) {
    using C2 = cplx<T>;
    using GE = Geo<T, N>;
    constexpr int CT = GE::CX5, G = GE::G, K = GE::K;
    constexpr int NBOX = GE::nbox(N), BR = GE::brows(N), BP = GE::bpitch(N, CT), RS = NBOX * BP;
    static_assert(NBOX == 1 || BR == BP, "x-forward staging must be contiguous in x");
    constexpr int KZP = KZP_, NTZ = KZP / CT;
    const int NTILE = kp.kyn * NTZ;   // tiles of this launch's ky rows
    constexpr uint32_t box_bytes = (uint32_t)(BR * CT * sizeof(C2));
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* S = reinterpret_cast<C2*>(smem_base128(smraw));   // [2][RS][CT]
    if (smem_u32(S) & 127u) {
        if (threadIdx.x == 0) atomicExch(err, 2);
        return;
    }
    // fields read: n (A fields 0..2), with the sponge first s (A fields 3..5),
    // whose sponge term -(1/C_sp) i k x s_hat/|k|^2 the n transforms add onto
    constexpr int NF = SP ? 6 : 3;
    auto field = [](int j) { return SP ? (j < 3 ? j + 3 : j - 3) : j; };
    C2* Rt = S + 2 * RS * CT;                             // [3][K][CT]
    C2* tw = Rt + 3 * K * CT;
    __shared__ __align__(8) uint64_t bar[2];
    const int col = threadIdx.x % CT, g = threadIdx.x / CT;
    const int mmax = kp.mmax, Kz = kp.Kz;
    const size_t FS = (size_t)K * K * KZP;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    using S3 = Split3<T, N>;
    const C2* tw3 = load_tw_split<T, N>(tw, twg, GE::tw_n);
    __syncthreads();
    auto issue = [&](int L) {  // one thread
        const int t = blockIdx.x + (L / NF) * gridDim.x, f = field(L % NF), buf = L & 1;
        if (t >= NTILE) return;
        const int cy = kp.ky0 + t / NTZ, czt = t % NTZ;
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar[buf], NBOX * box_bytes);
        for (int b = 0; b < NBOX; ++b)
            tma_load_2d(S + (size_t)(buf * RS + b * BP) * CT, &tm, 2 * czt * CT, (f * K + cy) * N + b * BR, &bar[buf]);
    };
    if (threadIdx.x == 0) issue(0);
    const T s = (T)kp.ks, sz = (T)kp.ksz;
    const T invn3 = (T)kp.invn3;
    const T dt = (T)kp.dt;
    int ti = 0;
    bool stop = false;
    constexpr int NBK = GE::nbox(K), BRK = GE::brows(K);
    for (int t = blockIdx.x; t < NTILE && !stop; t += gridDim.x, ++ti) {
        const int cy = kp.ky0 + t / NTZ, czt = t % NTZ;
        // U (first step) or Q of this tile is read only after the three
        // transforms: start pulling it into L2 now (measured: loading it into
        // registers here instead, held across the transforms, was slower)
        if (MODE == 0 && threadIdx.x < 3 * NBK) {
            const int f = threadIdx.x / NBK, b = threadIdx.x % NBK;
            tma_prefetch_2d(first ? &tmu : &tmh, 2 * czt * CT, (f * K + cy) * K + b * BRK);
        }
#pragma unroll 1
        for (int j = 0; j < NF; ++j) {
            const int L = NF * ti + j, buf = L & 1, f = field(j) % 3;
            const bool acc = SP && j >= 3;   // n onto the sponge term
            if (threadIdx.x == 0) issue(L + 1);
            const bool ok = mbar_wait(&bar[buf], (uint32_t)((L >> 1) & 1));
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) {
                    atomicExch(err, 1);
                    mbar_wait(&bar[buf ^ 1], (uint32_t)(((L + 1) >> 1) & 1));
                }
                stop = true;
                break;
            }
            C2* Sb = S + (size_t)buf * RS * CT;
            C2* Rf = Rt + f * K * CT;
            auto noload = [&](int) -> C2 { return cmk<C2>((T)0, (T)0); };
            if constexpr (S3::on) {
                // sub-line b = rows x = 3a + b, transformed in place; the kept
                // modes by the radix-3 recombination
                constexpr int M = S3::M;
                const int sub = g / S3::GM, gm = g % S3::GM;
                auto addr3 = [&](int p) { return (int)(Sb - S) + (3 * p + sub) * CT + col; };
                auto store = [&](int p, C2 v) { S[addr3(p)] = v; };
                LineFFT<T, M, -1>::template run<true>(S, tw, addr3, gm, noload, store);
                __syncthreads();
                for (int idx = threadIdx.x; idx < M * CT; idx += blockDim.x) {
                    const int kq = idx / CT, c = idx % CT;
                    C2 Zk, Zm;
                    split3_out(Sb[(3 * kq) * CT + c], Sb[(3 * kq + 1) * CT + c], Sb[(3 * kq + 2) * CT + c], tw3, kq,
                               M, Zk, Zm);
                    C2& r0 = Rf[kq * CT + c];                             // mode kq
                    r0 = acc ? cadd(r0, Zk) : Zk;
                    if (kq > 0) {                                          // mode kq - M
                        C2& r1 = Rf[(kq + M - 1) * CT + c];
                        r1 = acc ? cadd(r1, Zm) : Zm;
                    }
                }
            } else {
                auto addr = [&](int p) { return (int)(Sb - S) + p * CT + col; };
                auto store = [&](int q, C2 v) {
                    const int m = mode_of(q, N);
                    if (m <= mmax && m >= -mmax) {
                        C2& r = Rf[cidx_of(m, K) * CT + col];
                        r = acc ? cadd(r, v) : v;
                    }
                };
                LineFFT<T, N, -1>::template run<true>(S, tw, addr, g, noload, store);
            }
            __syncthreads();
            if constexpr (SP) {
                if (j == 2) {   // s_hat complete: replace it by the sponge term
                    const T myy = (T)cmode_of(cy, mmax, K);
                    for (int idx = threadIdx.x; idx < K * CT; idx += blockDim.x) {
                        const int cx = idx / CT, czz = czt * CT + idx % CT;
                        const int mx = cmode_of(cx, mmax, K);
                        const T kx = s * (T)mx, ky = s * myy, kz = sz * (T)czz;
                        const T k2 = kx * kx + ky * ky + kz * kz;
                        const C2 s0 = Rt[idx], s1 = Rt[K * CT + idx], s2 = Rt[2 * K * CT + idx];
                        const bool zero = (mx == 0 && cy == 0 && czz == 0);
                        const T fsp = zero ? (T)0 : -(T)kp.inv_csp / k2;
                        // i (k x s): (re, im) -> (-im, re)
                        const T ax = ky * s2.x - kz * s1.x, bx = ky * s2.y - kz * s1.y;
                        const T ay = kz * s0.x - kx * s2.x, by = kz * s0.y - kx * s2.y;
                        const T az = kx * s1.x - ky * s0.x, bz = kx * s1.y - ky * s0.y;
                        Rt[idx] = cmk<C2>(-fsp * bx, fsp * ax);
                        Rt[K * CT + idx] = cmk<C2>(-fsp * by, fsp * ay);
                        Rt[2 * K * CT + idx] = cmk<C2>(-fsp * bz, fsp * az);
                    }
                    __syncthreads();
                }
            }
        }
        if (stop) break;
        const T my = (T)cmode_of(cy, mmax, K);
        const T ey = Ex[cy];
        // projected nonlinear term of point idx (the 1/n^3 applied)
        auto proj = [&](int idx, int cx, int czz, C2* nn) {
            const int mx = cmode_of(cx, mmax, K);
            C2 n0 = Rt[idx], n1 = Rt[K * CT + idx], n2 = Rt[2 * K * CT + idx];
            n0.x *= invn3; n0.y *= invn3;
            n1.x *= invn3; n1.y *= invn3;
            n2.x *= invn3; n2.y *= invn3;
            const T kx = s * (T)mx, ky = s * my, kz = sz * (T)czz;
            const T k2 = kx * kx + ky * ky + kz * kz;
            const bool zero = (mx == 0 && cy == 0 && czz == 0);
            if (!zero) {
                const T ik2 = (T)1 / k2;
                const T dr = (kx * n0.x + ky * n1.x + kz * n2.x) * ik2;
                const T di = (kx * n0.y + ky * n1.y + kz * n2.y) * ik2;
                n0.x -= kx * dr; n0.y -= kx * di;
                n1.x -= ky * dr; n1.y -= ky * di;
                n2.x -= kz * dr; n2.y -= kz * di;
            } else if (MODE == 0 && !kp.mean_free) {
                n0 = n1 = n2 = cmk<C2>((T)0, (T)0);
            }
            nn[0] = n0; nn[1] = n1; nn[2] = n2;
        };
        // points per thread: every load of a point issued before its arithmetic
        constexpr int NT = CT * G, NPT = (K * CT + NT - 1) / NT;
#pragma unroll
        for (int r = 0; r < NPT; ++r) {
            const int idx = threadIdx.x + r * NT;
            const int cx = idx / CT, czz = czt * CT + idx % CT;
            if (idx >= K * CT || czz >= Kz) continue;
            const size_t o = ((size_t)cy * K + cx) * KZP + czz;
            C2 uq[3];
            if constexpr (MODE == 0) {
#pragma unroll
                for (int ff = 0; ff < 3; ++ff) uq[ff] = first ? U[ff * FS + o] : H[ff * FS + o];
            }
            if constexpr (MODE == 2) {
#pragma unroll
                for (int ff = 0; ff < 3; ++ff) {
                    const C2 v = Rt[ff * K * CT + idx];
                    U[ff * FS + o] = cmk<C2>(v.x * invn3, v.y * invn3);
                }
                continue;
            }
            if constexpr (MODE == 3) {   // Pi_hat = -i (k . N_hat) / |k|^2, Pi_hat(0) = 0
                const int mx = cmode_of(cx, mmax, K);
                const T kx = s * (T)mx, ky = s * my, kz = sz * (T)czz;
                const T k2 = kx * kx + ky * ky + kz * kz;
                const C2 n0 = Rt[idx], n1 = Rt[K * CT + idx], n2 = Rt[2 * K * CT + idx];
                const T dr = (kx * n0.x + ky * n1.x + kz * n2.x) * invn3;
                const T di = (kx * n0.y + ky * n1.y + kz * n2.y) * invn3;
                const bool zero = (mx == 0 && cy == 0 && czz == 0);
                const T ik2 = zero ? (T)0 : (T)1 / k2;
                U[o] = cmk<C2>(di * ik2, -dr * ik2);
                continue;
            }
            C2 nn[3];
            proj(idx, cx, czz, nn);
            if constexpr (MODE == 1) {
                U[o] = nn[0]; U[FS + o] = nn[1]; U[2 * FS + o] = nn[2];
                const C2 z = cmk<C2>((T)0, (T)0);
                H[o] = z; H[FS + o] = z; H[2 * FS + o] = z;
            } else {
                const T E = Ex[cx] * ey * Ez[czz];
#pragma unroll
                for (int ff = 0; ff < 3; ++ff) {
                    C2 un, qn;
                    ab2_update(uq[ff], nn[ff], E, dt, first != 0, un, qn);
                    U[ff * FS + o] = un;
                    H[ff * FS + o] = qn;
                }
            }
        }
        __syncthreads();
    }
}

// ----------------------------------------------- physical <-> z-spectral
// Persistent blocks over batches of L z lines (ZPhys): the batch's three
// fields arrive by bulk copies into one of two staging buffers while the
// block transforms the previous batch. Thread group r of line pair m (3 per
// pair, G threads each) runs one transform: r = 0, 1 the (u_x + i u_y) of
// line 2m + r, r = 2 the (u_z[2m] + i u_z[2m+1]). Template N is the z-line
// length (nz); there are kp.n^2 lines, a multiple of L. Every mbarrier wait
// is bounded: on timeout the kernel sets *err and stops.
//
// Forward: physical u (3 x n^3 real, [x][y][z]) -> B fields 0..2 (z r2c,
// kz < Kz).
template <typename T, int N>
__global__ void __launch_bounds__(ZPhys<T, N>::threads(ZPhys<T, N>::LF))
k_zfwd_phys(KP kp, const T* __restrict__ u, cplx<T>* __restrict__ B, const cplx<T>* __restrict__ twg,
            int* __restrict__ err) {
    using C2 = cplx<T>;
    using ZP = ZPhys<T, N>;
    constexpr int G = ZP::G, L = ZP::LF, LP = ZP::LP;
    constexpr bool WS = G <= 32 && 32 % G == 0;
    using FFT = LineFFT<T, N, -1, WS>;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* stage = reinterpret_cast<T*>(smem_base128(smraw));   // [2][3][L][N]
    if ((smem_u32(stage) & 127u) || (reinterpret_cast<uintptr_t>(u) & 15u)) {   // never expected
        if (threadIdx.x == 0) atomicExch(err, 2);
        return;
    }
    C2* tiles = reinterpret_cast<C2*>(stage + 2 * 3 * L * N);   // [3 L / 2][LP]
    C2* tw = tiles + 3 * (L / 2) * LP;
    __shared__ __align__(8) uint64_t bar[2];
    const int grp = threadIdx.x / G, g = threadIdx.x % G;
    const int m = grp / 3, r = grp % 3;
    const int Kz = kp.Kz, Kzp = kp.Kzp;
    const long nlines = (long)kp.n * kp.n;
    const int nb = (int)(nlines / L);
    const size_t BS = (size_t)nlines * Kzp;
    const size_t N3 = (size_t)nlines * N;
    constexpr uint32_t fbytes = (uint32_t)(L * N * sizeof(T));
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    load_tw(tw, twg, ZP::TWN);
    __syncthreads();
    auto issue = [&](int b, int buf) {  // one thread
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar[buf], 3 * fbytes);
#pragma unroll 1
        for (int f = 0; f < 3; ++f)
            bulk_g2s(stage + (size_t)(buf * 3 + f) * L * N, u + f * N3 + (size_t)b * L * N, fbytes, &bar[buf]);
    };
    if (threadIdx.x == 0 && (int)blockIdx.x < nb) issue(blockIdx.x, 0);
    C2* t = tiles + (size_t)grp * LP;
    const Pad16 addr{grp * LP};
    int it = 0;
    for (int b = blockIdx.x; b < nb; b += gridDim.x, ++it) {
        const int buf = it & 1;
        const bool more = b + (int)gridDim.x < nb;
        // the other buffer was read by the previous batch (end-of-batch barrier)
        if (threadIdx.x == 0 && more) issue(b + gridDim.x, buf ^ 1);
        const bool ok = mbar_wait(&bar[buf], (uint32_t)((it >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicExch(err, 1);
                if (more) mbar_wait(&bar[buf ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
            }
            break;
        }
        const T* st = stage + (size_t)buf * 3 * L * N;
        // r < 2: fields 0, 1 of line 2m + r; r = 2: field 2 of lines 2m, 2m + 1
        const T* s0 = r < 2 ? st + (size_t)(2 * m + r) * N : st + (size_t)(2 * L + 2 * m) * N;
        const T* s1 = r < 2 ? s0 + (size_t)L * N : s0 + N;
        auto load = [&](int z) -> C2 { return cmk<C2>(s0[z], s1[z]); };
        FFT::template run_tile<false>(tiles, tw, addr, g, load);
        // the transform's outputs are read back by other threads of the group
        if constexpr (WS) __syncwarp(warp_lanes());
        else __syncthreads();
        const size_t lo = ((size_t)b * L + 2 * m + (r == 1)) * Kzp;
        C2* oP = r < 2 ? B + lo : B + 2 * BS + lo;              // P = (Z_k + conj Z_{-k}) / 2
        C2* oQ = r < 2 ? B + BS + lo : B + 2 * BS + lo + Kzp;   // Q = (Z_k - conj Z_{-k}) / (2 i)
        for (int k = g; k < Kz; k += G) {
            const int mk = (N - k) % N;
            const C2 zk = t[k + (k >> 4)], zm = t[mk + (mk >> 4)];
            oP[k] = cmk<C2>((T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y));
            oQ[k] = cmk<C2>((T)0.5 * (zk.y + zm.y), (T)0.5 * (zm.x - zk.x));
        }
        __syncthreads();
    }
}

// Inverse: B fields 0..2 (z spectral, kz < Kz) -> physical u (3 x n^3 real).
template <typename T, int N>
__global__ void __launch_bounds__(ZPhys<T, N>::threads(ZPhys<T, N>::LI))
k_zinv_phys(KP kp, const cplx<T>* __restrict__ B, T* __restrict__ u, const cplx<T>* __restrict__ twg,
            int* __restrict__ err) {
    using C2 = cplx<T>;
    using ZP = ZPhys<T, N>;
    constexpr int G = ZP::G, L = ZP::LI, LP = ZP::LP, KZP = ZP::KZP;
    constexpr bool WS = G <= 32 && 32 % G == 0;
    using FFT = LineFFT<T, N, 1, WS>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* stage = reinterpret_cast<C2*>(smem_base128(smraw));   // [2][3][L][KZP]
    if (smem_u32(stage) & 127u) {   // never expected
        if (threadIdx.x == 0) atomicExch(err, 2);
        return;
    }
    C2* tiles = stage + 2 * 3 * L * KZP;   // [3 L / 2][LP]
    C2* tw = tiles + 3 * (L / 2) * LP;
    __shared__ __align__(8) uint64_t bar[2];
    const int grp = threadIdx.x / G, g = threadIdx.x % G;
    const int m = grp / 3, r = grp % 3;
    const int Kz = kp.Kz, Kzp = kp.Kzp;
    const long nlines = (long)kp.n * kp.n;
    const int nb = (int)(nlines / L);
    const size_t BS = (size_t)nlines * Kzp;
    const size_t N3 = (size_t)nlines * N;
    const uint32_t fbytes = (uint32_t)(L * Kzp * sizeof(C2));
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    load_tw(tw, twg, ZP::TWN);
    __syncthreads();
    auto issue = [&](int b, int buf) {  // one thread
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar[buf], 3 * fbytes);
#pragma unroll 1
        for (int f = 0; f < 3; ++f)
            bulk_g2s(stage + (size_t)(buf * 3 + f) * L * KZP, B + f * BS + (size_t)b * L * Kzp, fbytes, &bar[buf]);
    };
    if (threadIdx.x == 0 && (int)blockIdx.x < nb) issue(blockIdx.x, 0);
    const Pad16 addr{grp * LP};
    int it = 0;
    for (int b = blockIdx.x; b < nb; b += gridDim.x, ++it) {
        const int buf = it & 1;
        const bool more = b + (int)gridDim.x < nb;
        if (threadIdx.x == 0 && more) issue(b + gridDim.x, buf ^ 1);
        const bool ok = mbar_wait(&bar[buf], (uint32_t)((it >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicExch(err, 1);
                if (more) mbar_wait(&bar[buf ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
            }
            break;
        }
        const C2* st = stage + (size_t)buf * 3 * L * KZP;
        // r < 2: (A + i B) of fields 0, 1 of line 2m + r; r = 2: of field 2
        // of lines 2m and 2m + 1
        const C2* fa = r < 2 ? st + (size_t)(2 * m + r) * Kzp : st + (size_t)2 * L * KZP + (size_t)(2 * m) * Kzp;
        const C2* fb = r < 2 ? fa + (size_t)L * KZP : fa + Kzp;
        auto load = [&](int q) -> C2 {
            if (q < Kz) {
                C2 a = fa[q], c = fb[q];
                if (q == 0) { a.y = 0; c.y = 0; }
                return cmk<C2>(a.x - c.y, a.y + c.x);
            }
            if (q > N - Kz) {
                const C2 a = fa[N - q], c = fb[N - q];
                return cmk<C2>(a.x + c.y, c.x - a.y);
            }
            return cmk<C2>((T)0, (T)0);
        };
        const size_t po = ((size_t)b * L + 2 * m + (r == 1)) * N;
        T* o0 = r < 2 ? u + po : u + 2 * N3 + po;
        T* o1 = r < 2 ? u + N3 + po : u + 2 * N3 + po + N;
        auto store = [&](int z, C2 v) {
            o0[z] = v.x;
            o1[z] = v.y;
        };
        FFT::template run<false>(tiles, tw, addr, g, load, store);
        // the staging buffer and the tiles are reused by the next batches
        __syncthreads();
    }
}

// One field, B field 0 (z spectral) -> u[0..n^3) as u := (inverse) - u:
// persistent blocks over batches of L lines; a batch's L spectral lines and
// its L lines of u arrive by bulk copies into one of two staging buffers;
// thread group m (G threads) transforms the line pair (2m, 2m + 1) as one
// complex line. Bounded waits: on timeout the kernel sets *err and stops.
template <typename T, int N>
__global__ void __launch_bounds__(ZPhys<T, N>::threads_sub(ZPhys<T, N>::LS))
k_zinv_sub(KP kp, const cplx<T>* __restrict__ B, T* __restrict__ u, const cplx<T>* __restrict__ twg,
           int* __restrict__ err) {
    using C2 = cplx<T>;
    using ZP = ZPhys<T, N>;
    constexpr int G = ZP::G, L = ZP::LS, LP = ZP::LP, KZP = ZP::KZP;
    constexpr bool WS = G <= 32 && 32 % G == 0;
    using FFT = LineFFT<T, N, 1, WS>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* stage = reinterpret_cast<C2*>(smem_base128(smraw));   // [2][L][KZP] spectral
    T* ustage = reinterpret_cast<T*>(stage + 2 * L * KZP);     // [2][L][N] physical
    if ((smem_u32(stage) & 127u) || (reinterpret_cast<uintptr_t>(u) & 15u)) {   // never expected
        if (threadIdx.x == 0) atomicExch(err, 2);
        return;
    }
    C2* tiles = reinterpret_cast<C2*>(ustage + 2 * L * N);    // [L / 2][LP]
    C2* tw = tiles + (L / 2) * LP;
    __shared__ __align__(8) uint64_t bar[2];
    const int m = threadIdx.x / G, g = threadIdx.x % G;
    const int Kz = kp.Kz, Kzp = kp.Kzp;
    const long nlines = (long)kp.n * kp.n;
    const int nb = (int)(nlines / L);
    const uint32_t sbytes = (uint32_t)(L * Kzp * sizeof(C2));
    constexpr uint32_t ubytes = (uint32_t)(L * N * sizeof(T));
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    load_tw(tw, twg, ZP::TWN);
    __syncthreads();
    auto issue = [&](int b, int buf) {  // one thread
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar[buf], sbytes + ubytes);
        bulk_g2s(stage + (size_t)buf * L * KZP, B + (size_t)b * L * Kzp, sbytes, &bar[buf]);
        bulk_g2s(ustage + (size_t)buf * L * N, u + (size_t)b * L * N, ubytes, &bar[buf]);
    };
    if (threadIdx.x == 0 && (int)blockIdx.x < nb) issue(blockIdx.x, 0);
    const Pad16 addr{m * LP};
    int it = 0;
    for (int b = blockIdx.x; b < nb; b += gridDim.x, ++it) {
        const int buf = it & 1;
        const bool more = b + (int)gridDim.x < nb;
        if (threadIdx.x == 0 && more) issue(b + gridDim.x, buf ^ 1);
        const bool ok = mbar_wait(&bar[buf], (uint32_t)((it >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicExch(err, 1);
                if (more) mbar_wait(&bar[buf ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
            }
            break;
        }
        const C2* fa = stage + (size_t)buf * L * KZP + (size_t)(2 * m) * Kzp;
        const C2* fb = fa + Kzp;
        const T* su = ustage + (size_t)buf * L * N + (size_t)(2 * m) * N;
        // (A + i B) of the two real lines from their half spectra
        auto load = [&](int q) -> C2 {
            if (q < Kz) {
                C2 a = fa[q], c = fb[q];
                if (q == 0) { a.y = 0; c.y = 0; }
                return cmk<C2>(a.x - c.y, a.y + c.x);
            }
            if (q > N - Kz) {
                const C2 a = fa[N - q], c = fb[N - q];
                return cmk<C2>(a.x + c.y, c.x - a.y);
            }
            return cmk<C2>((T)0, (T)0);
        };
        T* o = u + ((size_t)b * L + 2 * m) * N;
        auto store = [&](int z, C2 v) {
            o[z] = v.x - su[z];
            o[N + z] = v.y - su[N + z];
        };
        FFT::template run<false>(tiles, tw, addr, g, load, store);
        // the staging buffer and the tiles are reused by the next batches
        __syncthreads();
    }
}

}  // namespace ps
