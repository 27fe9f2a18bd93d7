// ps_zstep.cuh -- pass 3 of the step (z c2r, n = u x omega - (chi/eta)(u - u_s),
// force/moment partial sums, z r2c) with u, omega and n kept in registers
// (Sec. 4.1, Eq. penalized Navier--Stokes; nonlinear term in physical space).
//
// Work unit: one sub-line of one z line (the whole line when n is not a
// multiple of 3; otherwise one of its three length-M sub-lines, M = n/3,
// see Split3), GL threads. A unit runs the three inverse transforms
// (u_x + i u_y), (u_z + i w_x), (w_y + i w_z) one after another: in a
// Stockham transform the positions a thread owns after the last stage
// (g + GL b + LsL u) are the positions its first-stage butterfly of a new
// transform of the same length needs (g + GL t), so the inverse outputs,
// the pointwise term at those positions and the first stage of the forward
// transforms never pass through shared memory. Units of lines 2m and 2m+1
// sit GL lanes apart in one warp: both write n_z into the pair's tile as
// the real and imaginary parts of (n_z[2m] + i n_z[2m+1]), which the even
// line's unit transforms forward. Forward
// outputs stay in the units' exchange tiles; one block-wide phase then does
// the radix-3 recombination of the sub-lines (n = 3M) and the two-for-one
// unpacking, and writes the kept z modes to B fields 0..2.
//
// Blocks are persistent over batches of LB consecutive lines; the six
// spectral lines of a batch arrive by bulk asynchronous copies (one staging
// buffer, refilled once the inverse transforms have read it). Every wait is
// bounded; on timeout the kernel records the error flag and stops.
#pragma once
#include "ps_kernels.cuh"

#ifndef PS_ZSTEP
#define PS_ZSTEP 1   // 1: the step's z pass is k_zstep where ZGeo::ok (FP32)
#endif
#ifndef PS_ZS_MINB
#define PS_ZS_MINB 0   // blocks per SM for the register budget (0: automatic)
#endif

namespace ps {

template <typename T, int N> struct ZGeo {
    using C2 = cplx<T>;
    static constexpr bool Z3 = (N % 3 == 0) && (PS_Z3 != 0);
    static constexpr int M = Z3 ? N / 3 : N;   // sub-line length
    static constexpr int NS = Z3 ? 3 : 1;      // sub-lines per line
    using FI = LineFFT<T, M, 1, true>;
    using FF = LineFFT<T, M, -1, true>;
    static constexpr int GL = FI::G;           // threads per unit
    static constexpr int SL = FI::SLOTS;       // transform outputs per thread
    static constexpr int MP = M + M / 16;      // padded exchange tile (zaddr padding)
    static constexpr int KZ = (N - 1) / 3 + 1;
    static constexpr int CW = 128 / (int)sizeof(C2);
    static constexpr int KZP = (KZ + CW - 1) / CW * CW;
    static constexpr int TWM = Z3 ? (tw_count(M) > 0 ? tw_count(M) : 1) : 0;
    static constexpr int NTW = Z3 ? TWM + 2 * M : (tw_count(N) > 0 ? tw_count(N) : 1);
    static constexpr int nt(int lb) { return NS * lb * GL; }
    static constexpr int lb_pick() {
        int l = 2;
        while ((nt(l) < 96 || nt(l) % 32 != 0) && l < 64) l *= 2;
        return l;
    }
    static constexpr int LB = lb_pick();       // lines per batch
    static constexpr int NT = nt(LB);          // threads per block
    static constexpr int smem() {
        return (int)sizeof(C2) * (6 * LB * KZP + (NS * LB + NS * LB / 2) * MP + NTW) + 6 * 8 * NT + 128;
    }
    // blocks per SM the register budget is sized for (four blocks of 96
    // threads: up to 168 registers per thread)
    static constexpr int MINB = PS_ZS_MINB > 0 ? PS_ZS_MINB : ((4 * NT * 128 <= 65536) ? 4 : 2);
    // units of lines 2m, 2m+1 share a warp (GL <= 16), exact last-stage
    // split, whole warps, FP32 (FP64 registers would not fit)
    static constexpr bool ok = sizeof(T) == 4 && GL <= 16 && 32 % GL == 0 &&
                               (FI::LsL % GL == 0 || FI::S == 1) && NT % 32 == 0 && NT <= 1024 &&
                               SL <= 16 && smem() <= 200 * 1024;
};

// Z[k] = F_0 + e^{-2 pi i k/n} F_1 + e^{-4 pi i k/n} F_2 (the low third of the
// kept modes) and Z[2M + k] (the high third) from the sub-line transforms.
template <typename C2>
__device__ __forceinline__ C2 split3_lo(C2 F0, C2 F1, C2 F2, const C2* tw3, int k, int M) {
    const C2 G1 = cmul(F1, cconj(tw3[k])), G2 = cmul(F2, cconj(tw3[M + k]));
    return cadd(F0, cadd(G1, G2));
}
template <typename C2>
__device__ __forceinline__ C2 split3_hi(C2 F0, C2 F1, C2 F2, const C2* tw3, int k, int M) {
    using T = typename real_of<C2>::type;
    const T h3 = (T)0.86602540378443864676;   // sin(2 pi / 3)
    const C2 G1 = cmul(F1, cconj(tw3[k])), G2 = cmul(F2, cconj(tw3[M + k]));
    return cmk<C2>(F0.x - (T)0.5 * (G1.x + G2.x) - h3 * (G1.y - G2.y),
                   F0.y - (T)0.5 * (G1.y + G2.y) + h3 * (G1.x - G2.x));
}

template <typename T, int N>
__global__ void __launch_bounds__(ZGeo<T, N>::NT, ZGeo<T, N>::MINB)
k_zstep(KP kp, cplx<T>* __restrict__ B, const T* __restrict__ chi, const T* __restrict__ us,
        const uint8_t* __restrict__ flag, double* __restrict__ partial, const cplx<T>* __restrict__ twg,
        int* __restrict__ err) {
    using C2 = cplx<T>;
    using ZG = ZGeo<T, N>;
    using FI = typename ZG::FI;
    using FF = typename ZG::FF;
    constexpr bool Z3 = ZG::Z3;
    constexpr int M = ZG::M, NS = ZG::NS, GL = ZG::GL, SL = ZG::SL, LB = ZG::LB, KZP = ZG::KZP, MP = ZG::MP;
    const int nyl = kp.n;   // lines per x-plane; the line length is N
    const int b0 = kp.xs0 * nyl / LB, b1 = (kp.xs0 + kp.xsn) * nyl / LB;   // this launch's batches
    constexpr uint32_t fbytes = (uint32_t)(LB * KZP * sizeof(C2));
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* stg = reinterpret_cast<C2*>(smem_base128(smraw));   // [6][LB][KZP]
    if (smem_u32(stg) & 127u) {   // never expected: refuse to start copies
        if (threadIdx.x == 0) atomicExch(err, 2);
        return;
    }
    C2* tiles = stg + 6 * LB * KZP;   // [NS LB] unit tiles, then [NS LB/2] n_z tiles, MP each
    C2* tw = tiles + (NS * LB + NS * LB / 2) * MP;
    // per-thread force/moment sums of the current batch (flagged lines only)
    double* fms = reinterpret_cast<double*>(tw + ZG::NTW) + 6 * threadIdx.x;
    __shared__ __align__(8) uint64_t bar;
    __shared__ double wacc[32][12];   // per-warp (sum, compensation) of the six sums
    // unit u = (sub (LB/2) + pair) 2 + side, line 2 pair + side
    const int unit = threadIdx.x / GL, g = threadIdx.x % GL;
    const int side = unit & 1, pair = (unit >> 1) % (LB / 2), sub = (unit >> 1) / (LB / 2);
    const int l = 2 * pair + side;
    C2* ut = tiles + unit * MP;
    C2* zt = tiles + (NS * LB + sub * (LB / 2) + pair) * MP;
    auto zad = [](int p) { return p + (p >> 4); };
    auto uaddr = [&](int p) { return (int)(ut - tiles) + zad(p); };
    auto zaddr_ = [&](int p) { return (int)(zt - tiles) + zad(p); };
    const int Kz = kp.Kz;
    const size_t BS = (size_t)nyl * nyl * KZP;
    const size_t N3 = (size_t)nyl * nyl * N;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    C2* tw3 = tw + ZG::TWM;   // n = 3M: e^{+2 pi i b q/n}, b = 1, 2
    if constexpr (Z3) {
        if constexpr (tw_count(M) > 0) load_tw(tw, twg + N, tw_count(M));
        load_tw(tw3, twg + 2 * N, 2 * M);
    } else {
        load_tw(tw, twg, ZG::NTW);
    }
    for (int i = threadIdx.x; i < 32 * 12; i += blockDim.x) (&wacc[0][0])[i] = 0.0;
    // slots of the force partials this launch does not reach stay zero
    if (blockIdx.x == 0)
        for (int i = (int)gridDim.x * 6 + threadIdx.x; i < kp.nparts * 6; i += blockDim.x)
            partial[(size_t)kp.part_off * 6 + i] = 0.0;
    __syncthreads();
    auto issue = [&](int bi) {   // one thread
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar, 6 * fbytes);
#pragma unroll 1
        for (int f = 0; f < 6; ++f)
            bulk_g2s(stg + (size_t)f * LB * KZP, B + f * BS + (size_t)bi * LB * KZP, fbytes, &bar);
    };
    if (threadIdx.x == 0 && b0 + (int)blockIdx.x < b1) issue(b0 + blockIdx.x);

    const T inv_eta = (T)kp.inv_eta;
    const T h3 = (T)0.86602540378443864676;   // sin(2 pi / 3)
    int it = 0;
    for (int bi = b0 + blockIdx.x; bi < b1; bi += gridDim.x, ++it) {
        const bool more = bi + (int)gridDim.x < b1;
        const bool ok = mbar_wait(&bar, (uint32_t)(it & 1));
        if (__syncthreads_or(!ok)) {
            // a copy never completed: record it, let the copy in flight land, stop
            if (threadIdx.x == 0) {
                atomicExch(err, 1);
                mbar_wait(&bar, (uint32_t)(it & 1));
            }
            break;
        }
        const long lid = (long)bi * LB + l;
        const bool flagged = flag[lid] != 0;
        const int x = (int)(lid / nyl), y = (int)(lid % nyl);
        C2 R0[SL], R1[SL];
        bool touched = false;
        if (flagged)
            for (int i = 0; i < 6; ++i) fms[i] = 0.0;
#pragma unroll 1
        for (int f = 0; f < 3; ++f) {
            const C2* fa = stg + (size_t)((2 * f) * LB + l) * KZP;
            const C2* fb = stg + (size_t)((2 * f + 1) * LB + l) * KZP;
            // input q of the (sub-)line transform from the two half spectra
            auto load = [&](int q) -> C2 {
                if constexpr (Z3) {
                    C2 a = fa[q], c = fb[q];
                    if (q == 0) { a.y = 0; c.y = 0; }
                    C2 v = cmk<C2>(a.x - c.y, a.y + c.x);                      // Z[q]
                    C2 w = cmk<C2>((T)0, (T)0);
                    if (q > 0) {
                        const C2 a2 = fa[M - q], c2 = fb[M - q];
                        w = cmk<C2>(a2.x + c2.y, c2.x - a2.y);                 // Z[q + 2M]
                    }
                    if (sub == 0) return cadd(v, w);
                    // e^{2 pi i 2 sub / 3}: sub 1 -> (-1/2, -h), sub 2 -> (-1/2, +h)
                    const T sg = sub == 1 ? -h3 : h3;
                    v = cmk<C2>(v.x - (T)0.5 * w.x - sg * w.y, v.y - (T)0.5 * w.y + sg * w.x);
                    return cmul(v, tw3[(sub - 1) * M + q]);
                } else {
                    if (q < Kz) {
                        C2 a = fa[q], c = fb[q];
                        if (q == 0) { a.y = 0; c.y = 0; }
                        return cmk<C2>(a.x - c.y, a.y + c.x);      // A + i B
                    }
                    if (q > N - Kz) {
                        const C2 a = fa[N - q], c = fb[N - q];
                        return cmk<C2>(a.x + c.y, c.x - a.y);      // conj(A) + i conj(B)
                    }
                    return cmk<C2>((T)0, (T)0);
                }
            };
            auto store = [&](int s, int p, C2 v) {
                if (f == 0) {
                    R0[s] = v;                              // u_x + i u_y
                } else if (f == 1) {
                    R1[s] = v;                              // u_z + i w_x
                } else {                                    // w_y + i w_z: n at this point
                    const T ux = R0[s].x, uy = R0[s].y, uz = R1[s].x, wx = R1[s].y, wy = v.x, wz = v.y;
                    T nx = uy * wz - uz * wy;
                    T ny = uz * wx - ux * wz;
                    T nzz = ux * wy - uy * wx;
                    if (flagged) {
                        const int z = Z3 ? 3 * p + sub : p;
                        const size_t po = (size_t)lid * N + z;
                        const T c = chi[po];
                        if (c != (T)0) {
                            const T sx = us[po], sy = us[N3 + po], sz = us[2 * N3 + po];
                            const T ce = c * inv_eta;
                            nx -= ce * (ux - sx);
                            ny -= ce * (uy - sy);
                            nzz -= ce * (uz - sz);
                            const double cd = (double)c;
                            const double px = cd * ((double)ux - (double)sx);
                            const double py = cd * ((double)uy - (double)sy);
                            const double pz = cd * ((double)uz - (double)sz);
                            const double rx = x * kp.dx - kp.x0[0], ry = y * kp.dx - kp.x0[1],
                                         rz = z * kp.dx - kp.x0[2];
                            fms[0] += px;
                            fms[1] += py;
                            fms[2] += pz;
                            fms[3] += ry * pz - rz * py;
                            fms[4] += rz * px - rx * pz;
                            fms[5] += rx * py - ry * px;
                            touched = true;
                        }
                    }
                    R0[s] = cmk<C2>(nx, ny);
                    // n_z into the pair's tile: even line real, odd line imaginary
                    T* zc = reinterpret_cast<T*>(tiles + zaddr_(p));
                    zc[side] = nzz;
                }
            };
            FI::template run_bu<false>(tiles, tw, uaddr, g, load, store);
            __syncwarp();   // the tile is read by the next transform's first stage
        }
        // every unit has read the staged spectra: the next batch may land
        __syncthreads();
        if (threadIdx.x == 0 && more) issue(bi + gridDim.x);
        // this batch's force sums: warp tree, then compensated into the warp slot
        if (__any_sync(0xffffffffu, touched)) {
            double fm[6];
            for (int i = 0; i < 6; ++i) fm[i] = flagged ? fms[i] : 0.0;
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
        // forward (n_x + i n_y) of this unit, outputs in place in its tile
        {
            auto load = [&](int t) -> C2 { return R0[FF::slot_of(t)]; };
            auto store = [&](int, int p, C2 v) { tiles[uaddr(p)] = v; };
            FF::run_regs_bu(tiles, tw, uaddr, g, load, store);
        }
        // forward (n_z[2m] + i n_z[2m+1]) by the even line's unit, from and
        // to the pair's tile (both units wrote it before the block barrier)
        {
            auto noload = [&](int) -> C2 { return cmk<C2>((T)0, (T)0); };
            auto store = [&](int p, C2 v) { tiles[zaddr_(p)] = v; };
            FF::template run_masked<true>(tiles, tw, zaddr_, g, noload, store, side == 0);
        }
        __syncthreads();
        // recombination (n = 3M) and two-for-one unpacking, kept kz < Kz;
        // per (line pair, k): both lines' fields 0, 1 and field 2
        for (int idx = threadIdx.x; idx < (LB / 2) * Kz; idx += blockDim.x) {
            const int pp = idx / Kz, k = idx % Kz;
            auto uz = [&](int b, int line) { return tiles + ((b * (LB / 2) + line / 2) * 2 + (line & 1)) * MP; };
            auto nzt = [&](int b) { return tiles + (NS * LB + b * (LB / 2) + pp) * MP; };
            // Z[k] and Z[n - k] of the transform whose sub-line tiles are t(b)
            auto zpair = [&](auto t, C2& zk, C2& zm) {
                if constexpr (Z3) {
                    const C2* t0 = t(0);
                    const C2* t1 = t(1);
                    const C2* t2 = t(2);
                    zk = split3_lo(t0[zad(k)], t1[zad(k)], t2[zad(k)], tw3, k, M);
                    if (k == 0) zm = zk;
                    else zm = split3_hi(t0[zad(M - k)], t1[zad(M - k)], t2[zad(M - k)], tw3, M - k, M);
                } else {
                    const C2* t0 = t(0);
                    zk = t0[zad(k)];
                    zm = t0[zad((N - k) % N)];
                }
            };
            // P = (Z_k + conj Z_{-k}) / 2,  Q = (Z_k - conj Z_{-k}) / (2 i)
            auto P = [](C2 zk, C2 zm) { return cmk<C2>((T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y)); };
            auto Q = [](C2 zk, C2 zm) { return cmk<C2>((T)0.5 * (zk.y + zm.y), (T)0.5 * (zm.x - zk.x)); };
#pragma unroll
            for (int sd = 0; sd < 2; ++sd) {
                const int line = 2 * pp + sd;
                C2 zk, zm;
                zpair([&](int b) { return uz(b, line); }, zk, zm);
                const size_t lo = ((size_t)bi * LB + line) * KZP;
                B[lo + k] = P(zk, zm);
                B[BS + lo + k] = Q(zk, zm);
            }
            C2 wk, wm;
            zpair(nzt, wk, wm);
            const size_t lo0 = ((size_t)bi * LB + 2 * pp) * KZP;
            B[2 * BS + lo0 + k] = P(wk, wm);
            B[2 * BS + lo0 + KZP + k] = Q(wk, wm);
        }
        __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        Acc a = {0, 0};
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) {
            a.add(wacc[w][2 * threadIdx.x]);
            a.add(wacc[w][2 * threadIdx.x + 1]);
        }
        partial[(size_t)(kp.part_off + blockIdx.x) * 6 + threadIdx.x] = a.val();
    }
}

}  // namespace ps
