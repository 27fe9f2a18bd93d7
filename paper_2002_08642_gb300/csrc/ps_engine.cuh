// ps_engine.cuh -- per-(precision, grid size) launch sequences of the step
// and of the physical <-> spectral conversions, behind a small table of
// function pointers so that the C ABI can dispatch on the runtime grid size.
#pragma once
#include "ps_kernels.cuh"

namespace ps {

struct Bufs {
    void* U;
    void* H;
    void* A;
    void* B;
    void* chi;
    void* us;
    uint8_t* flag;
    void* tw;        // twiddle table of the x/y/z lines (complex T)
    void* Ex;        // exp(-nu kx^2 dt) for the K x/y modes (T)
    void* Ez;        // exp(-nu kz^2 dt) for the Kz z modes (T)
    double* partial; // per-block partial sums
    int* err;        // device error flag (bounded waits that gave up)
    const CUtensorMap* tmA;  // A as {2 Kzp reals, n rows, 6 K planes} (y-inverse input)
    const CUtensorMap* tmB;  // B as rows of 2 Kzp reals (y-forward input)
    const CUtensorMap* tmU;  // U as rows of 2 Kzp reals (x-inverse input)
    const CUtensorMap* tmA5; // A as rows of 2 Kzp reals (x-forward input)
    const CUtensorMap* tmUp; // U, H as rows of 2 Kzp reals, x-forward box (L2 prefetch)
    const CUtensorMap* tmHp;
    const CUtensorMap* tmG;  // adjoint G as rows of 2 Kzp reals, x-inverse box (null without adjoint)
    const void* chi_sp;      // sponge mask (n^3, caller-owned), null when the sponge term is off
    void* N3;                // keep_uw: 3 z-spectral fields [f][x][y][kz] for the pressure's N (else null)
    const CUtensorMap* tmN;  // N3 as rows of 2 Kzp reals (y-forward input), keep_uw only
};

// Timing events of one step: start/end of P1, P2, P3, P4, P5.
static constexpr int kEvPerStep = 10;

struct Ops {
    int n, nz, C, C5, G;
    int cy2, br2, cy4, br4;   // TMA box widths (complex) and heights of the y passes
    int cx1, cx5;             // TMA box widths of the x passes (heights br2, br4)
    int zblocks;  // blocks of the z pass (= number of force partials), set by prepare
    cudaError_t (*prepare)(int nsm, int* zblocks);
    // ev (nullable): kEvPerStep events (see kEvPerStep)
    cudaError_t (*step)(const KP&, const Bufs&, int first, int resume, cudaStream_t, cudaEvent_t* ev);
    cudaError_t (*set_velocity)(const KP&, const Bufs&, const void* u, cudaStream_t);
    cudaError_t (*get_velocity)(const KP&, const Bufs&, void* u, cudaStream_t);
    // generic 3-field transforms between compact spectral arrays (3 x
    // [ky][kx][kz]) and physical arrays (3 x n^3); A, B are used as scratch
    cudaError_t (*inv3)(const KP&, const Bufs&, const void* spec, void* phys, cudaStream_t);
    cudaError_t (*fwd3)(const KP&, const Bufs&, const void* phys, void* spec, cudaStream_t);
    // physical u and omega of the state in U (A, B used as scratch)
    cudaError_t (*inv_uw)(const KP&, const Bufs&, void* u, void* w, cudaStream_t);
    // physical inverse of the adjoint array G (needs b.tmG)
    cudaError_t (*inv_g)(const KP&, const Bufs&, void* phys, cudaStream_t);
    // static pressure of the state in U with the current mask (n^3 real)
    cudaError_t (*pressure)(const KP&, const Bufs&, void* p, int resume, cudaStream_t);
    // one phase of the step on a slab (kp.xs0/xsn x-planes, kp.ky0/kyn ky
    // rows): 0 x-inverse + curl on the ky rows; 1 y-inverse, z pass and
    // y-forward on the x-planes; 2 x-forward, projection and update on the
    // ky rows. The x-planes of a slab start and end at multiples of zalign/n.
    cudaError_t (*slab_phase)(const KP&, const Bufs&, int phase, int first, cudaStream_t);
    int zalign;   // z lines per z-pass batch (slab boundaries x n must be multiples)
};

// N x N x NZ grid: the x and y passes are the kernels of length-N lines,
// the z passes those of length-NZ lines (NZ = N, or N/2 for the 4 x 4 x 2
// box); the z kernels take N at run time, so both grids share them.
template <typename T, int N, int NZ = N> struct Engine {
    using C2 = cplx<T>;
    using GE = Geo<T, N>;
    using GZ = Geo<T, NZ>;
    static constexpr int KZ_ = GZ::KZP;   // kz columns (compile-time in the x/y passes)
    static constexpr size_t tw_bytes = (size_t)GE::tw_n * sizeof(C2);
    static constexpr size_t sm_strided = tw_bytes + (size_t)N * GE::C * sizeof(C2);
    static constexpr size_t sm_x5 = tw_bytes + (size_t)3 * N * GE::C5 * sizeof(C2);
    static constexpr size_t sm_zp = (size_t)GZ::zsmem(GZ::LZ);
    static constexpr int thr_s = GE::C * GE::G;
    static constexpr int thr_5 = GE::C5 * GE::G;
    static constexpr int thr_zp = 3 * GZ::LZ * GZ::G;
    // persistent physical <-> z-spectral transforms
    using ZP = ZPhys<T, NZ>;
    static constexpr size_t sm_zi = (size_t)ZP::smem(ZP::LI, false);
    static constexpr size_t sm_zf = (size_t)ZP::smem(ZP::LF, true);
    static constexpr int thr_zi = ZP::threads(ZP::LI);
    static constexpr int thr_zf = ZP::threads(ZP::LF);
    static constexpr size_t sm_zs = (size_t)ZP::smem_sub(ZP::LS);
    static constexpr int thr_zs = ZP::threads_sub(ZP::LS);
    static_assert((N * N) % ZP::LI == 0 && (N * N) % ZP::LF == 0 && (N * N) % ZP::LS == 0,
                  "z-line batches divide the lines");
    static int& zigrid() {
        static int g = 0;
        return g;
    }
    static int& zfgrid() {
        static int g = 0;
        return g;
    }
    static int& zsgrid() {
        static int g = 0;
        return g;
    }
    // twiddles of the z lines: the table of length-NZ lines sits after the
    // length-N one when the lengths differ
    static const C2* twz(const void* tw) { return (const C2*)tw + (NZ == N ? 0 : 3 * N); }

    template <class K> static cudaError_t attr(K k, size_t bytes) {
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    }

    static int& zgrid() {  // persistent z-pass blocks (set by prepare)
        static int g = 0;
        return g;
    }

    static int& y2grid() {
        static int g = 0;
        return g;
    }
    static int& y4grid() {
        static int g = 0;
        return g;
    }
    static int& x1grid() {
        static int g = 0;
        return g;
    }
    static int& x5grid() {
        static int g = 0;
        return g;
    }
    static constexpr size_t sm_x1 = (size_t)GE::y2_smem(GE::CX1);
    static constexpr size_t sm_x5t = (size_t)GE::x5_smem(GE::CX5);
    static constexpr size_t sm_x5s = sm_x5t;   // the sponge variant keeps three result tiles
    static int& x5sgrid() {
        static int g = 0;
        return g;
    }
    static constexpr int thr_x1 = GE::CX1 * GE::G;
    static constexpr int thr_x5 = GE::CX5 * GE::G;
    static constexpr size_t sm_y2 = (size_t)GE::y2_smem(GE::CY2, GE::Y2NB);
    static constexpr size_t sm_y4 = (size_t)GE::y4_smem(GE::CY4);
    static constexpr int thr_y2 = GE::CY2 * GE::G;
    static constexpr int thr_y4 = GE::CY4 * GE::G;

    static cudaError_t prepare(int nsm, int* zb) {
        cudaError_t e;
        if ((e = attr(k_xinv<T, N, 6>, sm_strided))) return e;
        if ((e = attr(k_xinv<T, N, 3>, sm_strided))) return e;
        if ((e = attr(k_yinv<T, N, 6>, sm_strided))) return e;
        if ((e = attr(k_yinv<T, N, 3>, sm_strided))) return e;
        if ((e = attr(k_yfwd<T, N>, sm_strided))) return e;
        if ((e = attr(k_zpass<T, NZ, false, false, N>, sm_zp))) return e;
        if ((e = attr(k_zpass<T, NZ, true, false, N>, sm_zp))) return e;
        if ((e = attr(k_xinv<T, N, 1>, sm_strided))) return e;
        if ((e = attr(k_yinv<T, N, 1>, sm_strided))) return e;
        if ((e = attr(k_zinv_sub<T, NZ>, sm_zs))) return e;
        if ((e = attr(k_zfwd_phys<T, NZ>, sm_zf))) return e;
        if ((e = attr(k_zinv_phys<T, NZ>, sm_zi))) return e;
        if ((e = attr(k_xfwd<T, N, 0>, sm_x5))) return e;
        if ((e = attr(k_xfwd<T, N, 1>, sm_x5))) return e;
        if ((e = attr(k_xfwd<T, N, 2>, sm_x5))) return e;
        int occ = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_zpass<T, NZ, false, false, N>, thr_zp, sm_zp))) return e;
        if (occ < 1) occ = 1;
        const int nb = N * N / GZ::LZ;
        zgrid() = nsm * occ < nb ? nsm * occ : nb;
        *zb = zgrid();

        if ((e = attr(k_yinv_tma<T, N, 6, KZ_>, sm_y2))) return e;
        if ((e = attr(k_yfwd_tma<T, N, GE::CY4, 3, KZ_>, sm_y4))) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_yinv_tma<T, N, 6, KZ_>, thr_y2, sm_y2))) return e;
        y2grid() = nsm * (occ < 1 ? 1 : occ);
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_yfwd_tma<T, N, GE::CY4, 3, KZ_>, thr_y4, sm_y4))) return e;
        y4grid() = nsm * (occ < 1 ? 1 : occ);
        if ((e = attr(k_xinv_tma<T, N, 6, KZ_>, sm_x1))) return e;
        if ((e = attr(k_xinv_tma<T, N, 3, KZ_>, sm_x1))) return e;
        if ((e = attr(k_yinv_tma<T, N, 3, KZ_>, sm_y2))) return e;
        if ((e = attr(k_yinv_tma<T, N, 1, KZ_>, sm_y2))) return e;
        if ((e = attr(k_xfwd_tma<T, N, 0, false, KZ_>, sm_x5t))) return e;
        if ((e = attr(k_xfwd_tma<T, N, 1, false, KZ_>, sm_x5t))) return e;
        if ((e = attr(k_xfwd_tma<T, N, 2, false, KZ_>, sm_x5t))) return e;
        if ((e = attr(k_xfwd_tma<T, N, 3, false, KZ_>, sm_x5t))) return e;
        if ((e = attr(k_xfwd_tma<T, N, 0, true, KZ_>, sm_x5s))) return e;
        if ((e = attr(k_zpass<T, NZ, false, true, N>, sm_zp))) return e;
        if ((e = attr(k_yfwd_tma<T, N, GE::CY4, 6, KZ_>, sm_y4))) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_xfwd_tma<T, N, 0, true, KZ_>, thr_x5, sm_x5s)))
            return e;
        x5sgrid() = nsm * (occ < 1 ? 1 : occ);
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_xinv_tma<T, N, 6, KZ_>, thr_x1, sm_x1))) return e;
        x1grid() = nsm * (occ < 1 ? 1 : occ);
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_xfwd_tma<T, N, 0, false, KZ_>, thr_x5, sm_x5t))) return e;
        x5grid() = nsm * (occ < 1 ? 1 : occ);
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_zinv_phys<T, NZ>, thr_zi, sm_zi))) return e;
        zigrid() = nsm * (occ < 1 ? 1 : occ);
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_zfwd_phys<T, NZ>, thr_zf, sm_zf))) return e;
        zfgrid() = nsm * (occ < 1 ? 1 : occ);
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_zinv_sub<T, NZ>, thr_zs, sm_zs))) return e;
        zsgrid() = nsm * (occ < 1 ? 1 : occ);
        return cudaSuccess;
    }

    static dim3 grid_xs(const KP& kp, int C) { return dim3(kp.Kzp / C, kp.K); }
    static dim3 grid_ys(const KP& kp) { return dim3(kp.Kzp / GE::C, N); }


    // resume: B already holds u and omega of the state (y-inverse output,
    // left by the pressure evaluation of a keep_uw context), so passes 1 and
    // 2 are skipped; their timing events are recorded back to back
    static cudaError_t step(const KP& kp, const Bufs& b, int first, int resume, cudaStream_t s, cudaEvent_t* ev) {
        const C2* tw = (const C2*)b.tw;
        KP k1 = kp;
        k1.xs0 = 0; k1.xsn = N; k1.part_off = 0;
        const bool sp = b.chi_sp != nullptr;   // sponge term: six-field z/y-forward variants
        if (ev) cudaEventRecord(ev[0], s);
        if (!resume) k_xinv_tma<T, N, 6, KZ_><<<x1grid(), thr_x1, sm_x1, s>>>(*b.tmU, kp, (C2*)b.A, tw, b.err);
        if (ev) { cudaEventRecord(ev[1], s); cudaEventRecord(ev[2], s); }
        if (!resume) k_yinv_tma<T, N, 6, KZ_><<<y2grid(), thr_y2, sm_y2, s>>>(*b.tmA, k1, (C2*)b.B, tw, b.err);
        if (ev) { cudaEventRecord(ev[3], s); cudaEventRecord(ev[4], s); }
        if (sp)
            k_zpass<T, NZ, false, true, N><<<zgrid(), thr_zp, sm_zp, s>>>(k1, (C2*)b.B, (const T*)b.chi, (const T*)b.us,
                                                                     b.flag, b.partial, twz(b.tw), b.err, nullptr,
                                                                     (const T*)b.chi_sp, (C2*)b.B);
        else
            k_zpass<T, NZ, false, false, N><<<zgrid(), thr_zp, sm_zp, s>>>(k1, (C2*)b.B, (const T*)b.chi, (const T*)b.us, b.flag,
                                                        b.partial, twz(b.tw), b.err, nullptr, nullptr, (C2*)b.B);
        if (ev) { cudaEventRecord(ev[5], s); cudaEventRecord(ev[6], s); }
        if (sp) k_yfwd_tma<T, N, GE::CY4, 6, KZ_><<<y4grid(), thr_y4, sm_y4, s>>>(*b.tmB, k1, (C2*)b.A, tw, b.err);
        else k_yfwd_tma<T, N, GE::CY4, 3, KZ_><<<y4grid(), thr_y4, sm_y4, s>>>(*b.tmB, k1, (C2*)b.A, tw, b.err);
        if (ev) { cudaEventRecord(ev[7], s); cudaEventRecord(ev[8], s); }
        if (sp)
            k_xfwd_tma<T, N, 0, true, KZ_><<<x5sgrid(), thr_x5, sm_x5s, s>>>(*b.tmA5, *b.tmUp, *b.tmHp, kp, (C2*)b.U,
                                                                       (C2*)b.H, (const T*)b.Ex, (const T*)b.Ez,
                                                                       first, tw, b.err);
        else
            k_xfwd_tma<T, N, 0, false, KZ_><<<x5grid(), thr_x5, sm_x5t, s>>>(*b.tmA5, *b.tmUp, *b.tmHp, kp, (C2*)b.U,
                                                                (C2*)b.H, (const T*)b.Ex, (const T*)b.Ez, first, tw,
                                                                b.err);
        if (ev) cudaEventRecord(ev[9], s);
        return cudaGetLastError();
    }

    static cudaError_t set_velocity(const KP& kp, const Bufs& b, const void* u, cudaStream_t s) {
        const C2* tw = (const C2*)b.tw;
        k_zfwd_phys<T, NZ><<<zfgrid(), thr_zf, sm_zf, s>>>(kp, (const T*)u, (C2*)b.B, twz(b.tw), b.err);
        k_yfwd<T, N><<<grid_ys(kp), thr_s, sm_strided, s>>>(kp, (const C2*)b.B, (C2*)b.A, tw);
        k_xfwd_tma<T, N, 1, false, KZ_><<<x5grid(), thr_x5, sm_x5t, s>>>(*b.tmA5, *b.tmUp, *b.tmHp, kp, (C2*)b.U, (C2*)b.H,
                                                            (const T*)b.Ex, (const T*)b.Ez, 0, tw, b.err);
        return cudaGetLastError();
    }

    static cudaError_t get_velocity(const KP& kp, const Bufs& b, void* u, cudaStream_t s) {
        const C2* tw = (const C2*)b.tw;
        k_xinv<T, N, 3><<<grid_xs(kp, GE::C), thr_s, sm_strided, s>>>(kp, (const C2*)b.U, (C2*)b.A, tw);
        k_yinv<T, N, 3><<<grid_ys(kp), thr_s, sm_strided, s>>>(kp, (const C2*)b.A, (C2*)b.B, tw);
        k_zinv_phys<T, NZ><<<zigrid(), thr_zi, sm_zi, s>>>(kp, (const C2*)b.B, (T*)u, twz(b.tw), b.err);
        return cudaGetLastError();
    }

    static cudaError_t inv3(const KP& kp, const Bufs& b, const void* spec, void* phys, cudaStream_t s) {
        const C2* tw = (const C2*)b.tw;
        k_xinv<T, N, 3><<<grid_xs(kp, GE::C), thr_s, sm_strided, s>>>(kp, (const C2*)spec, (C2*)b.A, tw);
        k_yinv<T, N, 3><<<grid_ys(kp), thr_s, sm_strided, s>>>(kp, (const C2*)b.A, (C2*)b.B, tw);
        k_zinv_phys<T, NZ><<<zigrid(), thr_zi, sm_zi, s>>>(kp, (const C2*)b.B, (T*)phys, twz(b.tw), b.err);
        return cudaGetLastError();
    }

    static cudaError_t fwd3(const KP& kp, const Bufs& b, const void* phys, void* spec, cudaStream_t s) {
        const C2* tw = (const C2*)b.tw;
        KP k1 = kp;
        k1.xs0 = 0; k1.xsn = N; k1.part_off = 0;
        k_zfwd_phys<T, NZ><<<zfgrid(), thr_zf, sm_zf, s>>>(k1, (const T*)phys, (C2*)b.B, twz(b.tw), b.err);
        k_yfwd_tma<T, N, GE::CY4, 3, KZ_><<<y4grid(), thr_y4, sm_y4, s>>>(*b.tmB, k1, (C2*)b.A, tw, b.err);
        k_xfwd_tma<T, N, 2, false, KZ_><<<x5grid(), thr_x5, sm_x5t, s>>>(*b.tmA5, *b.tmUp, *b.tmHp, k1, (C2*)spec, nullptr,
                                                            (const T*)b.Ex, (const T*)b.Ez, 0, tw, b.err);
        return cudaGetLastError();
    }

    // physical (3 x n^3) inverse transform of the adjoint array G (b.tmG)
    // through the TMA x and y passes
    static cudaError_t inv_g(const KP& kp, const Bufs& b, void* phys, cudaStream_t s) {
        const C2* tw = (const C2*)b.tw;
        KP k1 = kp;
        k1.xs0 = 0; k1.xsn = N; k1.part_off = 0;
        k_xinv_tma<T, N, 3, KZ_><<<x1grid(), thr_x1, sm_x1, s>>>(*b.tmG, k1, (C2*)b.A, tw, b.err);
        k_yinv_tma<T, N, 3, KZ_><<<y2grid(), thr_y2, sm_y2, s>>>(*b.tmA, k1, (C2*)b.B, tw, b.err);
        k_zinv_phys<T, NZ><<<zigrid(), thr_zi, sm_zi, s>>>(k1, (const C2*)b.B, (T*)phys, twz(b.tw), b.err);
        return cudaGetLastError();
    }

    // static pressure p = Pi - (1/2)|u|^2 of the state U with the current
    // mask (n^3, [x][y][z]): the step's passes 1-4 (the z pass also writing
    // (1/2)|u|^2 to p), the x-forward pass writing Pi_hat into A's field 3,
    // then its inverse (x; y by the TMA-staged pass; z pairs of lines:
    // p := Pi - p)
    // With b.N3 (keep_uw) the z pass writes N to N3 and the inverse of Pi
    // runs through A and N3, so B still holds u and omega of the state at
    // the end: the next step may resume at its z pass. resume: B already
    // holds them (a second evaluation on the same state), skip passes 1-2.
    static cudaError_t pressure(const KP& kp, const Bufs& b, void* p, int resume, cudaStream_t s) {
        const C2* tw = (const C2*)b.tw;
        KP k1 = kp;
        k1.xs0 = 0; k1.xsn = N; k1.part_off = 0;
        if (!resume) {
            k_xinv_tma<T, N, 6, KZ_><<<x1grid(), thr_x1, sm_x1, s>>>(*b.tmU, k1, (C2*)b.A, tw, b.err);
            k_yinv_tma<T, N, 6, KZ_><<<y2grid(), thr_y2, sm_y2, s>>>(*b.tmA, k1, (C2*)b.B, tw, b.err);
        }
        C2* nout = b.N3 ? (C2*)b.N3 : (C2*)b.B;
        k_zpass<T, NZ, true, false, N><<<zgrid(), thr_zp, sm_zp, s>>>(k1, (C2*)b.B, (const T*)b.chi, (const T*)b.us, b.flag,
                                                          b.partial, twz(b.tw), b.err, (T*)p, nullptr, nout);
        k_yfwd_tma<T, N, GE::CY4, 3, KZ_><<<y4grid(), thr_y4, sm_y4, s>>>(b.N3 ? *b.tmN : *b.tmB, k1, (C2*)b.A, tw,
                                                                  b.err);
        C2* pih = (C2*)b.A + (size_t)3 * N * GE::K * kp.Kzp;
        k_xfwd_tma<T, N, 3, false, KZ_><<<x5grid(), thr_x5, sm_x5t, s>>>(*b.tmA5, *b.tmUp, *b.tmHp, k1, pih, nullptr,
                                                            (const T*)b.Ex, (const T*)b.Ez, 0, tw, b.err);
        k_xinv<T, N, 1><<<grid_xs(k1, GE::C), thr_s, sm_strided, s>>>(k1, pih, (C2*)b.A, tw);
        k_yinv_tma<T, N, 1, KZ_><<<y2grid(), thr_y2, sm_y2, s>>>(*b.tmA, k1, nout, tw, b.err);
        k_zinv_sub<T, NZ><<<zsgrid(), thr_zs, sm_zs, s>>>(k1, (const C2*)nout, (T*)p, twz(b.tw), b.err);
        return cudaGetLastError();
    }

    // u and omega = curl u of the state U, physical (3 x n^3 each): the
    // step's x (curl fused) and y passes, then z c2r of fields 0..2 and 3..5
    static cudaError_t inv_uw(const KP& kp, const Bufs& b, void* u, void* w, cudaStream_t s) {
        const C2* tw = (const C2*)b.tw;
        KP k1 = kp;
        k1.xs0 = 0; k1.xsn = N; k1.part_off = 0;
        k_xinv_tma<T, N, 6, KZ_><<<x1grid(), thr_x1, sm_x1, s>>>(*b.tmU, k1, (C2*)b.A, tw, b.err);
        k_yinv_tma<T, N, 6, KZ_><<<y2grid(), thr_y2, sm_y2, s>>>(*b.tmA, k1, (C2*)b.B, tw, b.err);
        const size_t BS = (size_t)N * N * k1.Kzp;
        k_zinv_phys<T, NZ><<<zigrid(), thr_zi, sm_zi, s>>>(k1, (const C2*)b.B, (T*)u, twz(b.tw), b.err);
        k_zinv_phys<T, NZ><<<zigrid(), thr_zi, sm_zi, s>>>(k1, (const C2*)b.B + 3 * BS, (T*)w, twz(b.tw), b.err);
        return cudaGetLastError();
    }

    static cudaError_t slab_phase(const KP& kp, const Bufs& b, int phase, int first, cudaStream_t s) {
        const C2* tw = (const C2*)b.tw;
        if (phase == 0) {
            k_xinv_tma<T, N, 6, KZ_><<<x1grid(), thr_x1, sm_x1, s>>>(*b.tmU, kp, (C2*)b.A, tw, b.err);
        } else if (phase == 1) {
            k_yinv_tma<T, N, 6, KZ_><<<y2grid(), thr_y2, sm_y2, s>>>(*b.tmA, kp, (C2*)b.B, tw, b.err);
            k_zpass<T, NZ, false, false, N><<<zgrid(), thr_zp, sm_zp, s>>>(kp, (C2*)b.B, (const T*)b.chi, (const T*)b.us, b.flag,
                                                        b.partial, twz(b.tw), b.err, nullptr, nullptr, (C2*)b.B);
            k_yfwd_tma<T, N, GE::CY4, 3, KZ_><<<y4grid(), thr_y4, sm_y4, s>>>(*b.tmB, kp, (C2*)b.A, tw, b.err);
        } else {
            k_xfwd_tma<T, N, 0, false, KZ_><<<x5grid(), thr_x5, sm_x5t, s>>>(*b.tmA5, *b.tmUp, *b.tmHp, kp, (C2*)b.U,
                                                                (C2*)b.H, (const T*)b.Ex, (const T*)b.Ez, first, tw,
                                                                b.err);
        }
        return cudaGetLastError();
    }

    static Ops ops() {
        Ops o;
        o.n = N; o.nz = NZ; o.C = GE::C; o.C5 = GE::C5; o.G = GE::G;
        o.cy2 = GE::CY2; o.br2 = GE::brows(GE::K); o.cy4 = GE::CY4; o.br4 = GE::brows(N);
        o.cx1 = GE::CX1; o.cx5 = GE::CX5;
        o.zblocks = 0;
        o.prepare = &prepare;
        o.step = &step;
        o.set_velocity = &set_velocity;
        o.get_velocity = &get_velocity;
        o.inv3 = &inv3;
        o.fwd3 = &fwd3;
        o.inv_uw = &inv_uw;
        o.inv_g = &inv_g;
        o.pressure = &pressure;
        o.slab_phase = &slab_phase;
        o.zalign = GZ::LZ;
        return o;
    }
};

// Grid sizes built into the library, as two halving chains so that every
// N x N x N/2 engine is compiled in the translation unit that holds the
// kernels of both of its line lengths.
#define PS_SIZES_A(X) X(12) X(24) X(48) X(96) X(192) X(384) X(768)
#define PS_SIZES_B(X) X(16) X(32) X(64) X(128) X(256) X(512)
#define PS_SIZES(X) PS_SIZES_A(X) PS_SIZES_B(X)
// smallest n with an N x N x N/2 engine
static constexpr int kMinAnisoN = 32;

// Engine of an n x n x nz grid of the built sizes (nz = n, or n/2 for
// n >= kMinAnisoN), else null.
template <typename T, int N> const Ops* ops_for_nz(int nz) {
    if (nz == N) {
        static const Ops o = Engine<T, N>::ops();
        return &o;
    }
    if constexpr (N >= kMinAnisoN) {
        if (2 * nz == N) {
            static const Ops o = Engine<T, N, N / 2>::ops();
            return &o;
        }
    }
    return nullptr;
}

// Defined in the per-precision, per-chain translation units.
const Ops* ops_f32_a(int n, int nz);
const Ops* ops_f32_b(int n, int nz);
const Ops* ops_f64_a(int n, int nz);
const Ops* ops_f64_b(int n, int nz);

}  // namespace ps
