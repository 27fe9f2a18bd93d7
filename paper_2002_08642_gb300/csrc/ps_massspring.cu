// ps_massspring.cu -- host mass-spring network of the wing (Sec. 2.1-2.2:
// extension and bending springs, Eq. extension_spring, Eq.
// two_bending_angles; Newton's law in first-order form, Eq.
// Newton_law_first_order, advanced by variable-step BDF2, Eq.
// discretized_ODEs, with Newton--Raphson). Host code: the network has
// hundreds to a few thousand nodes; the GPU rasteriser and the pressure-load
// kernel take its node positions and return its external forces.
//
// Energy E = sum_ext (1/2) k^e (|x_j - x_i| - l_0)^2
//          + sum_bend (1/2) k^b [(theta^y - theta^y_0)^2 + (theta^z - theta^z_0)^2],
// theta^y = atan2(A, B), A = a_x b_y - b_x a_y, B = a_x b_x + a_y b_y
// (a = x_j - x_i, b = x_k - x_j; theta^z with z for y; angle changes taken
// in (-pi, pi]). Internal forces are -grad E in closed form: the extension
// force is the printed one, the bending force is the gradient of the
// bending energy (the printed bending force has no lever length; the k^b -
// EI relation of Eq. EI_k_relation equates energies, which this keeps).
//
// Newton matrix: the extension springs' stiffness in closed form, the
// bending springs' by central differences of each spring's own 9 force
// components, assembled on the free nodes in reverse Cuthill--McKee order
// into a band matrix and solved by banded LU with partial pivoting.
// Solving in a moving frame adds the fictitious forces
// -m (A_O + dOmega x x + Omega x (Omega x x) + 2 Omega x v), implicit like
// the spring forces.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "ps.h"
#include "ps_fault.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

struct Ext { int i, j; double k, l0; };
struct Bend { int i, j, k; double kb, t0y, t0z; };

double wrap(double d) {   // into (-pi, pi]
    while (d > kPi) d -= 2.0 * kPi;
    while (d <= -kPi) d += 2.0 * kPi;
    return d;
}

void bend_angles(const double* xi, const double* xj, const double* xk, double* ty, double* tz) {
    const double a[3] = {xj[0] - xi[0], xj[1] - xi[1], xj[2] - xi[2]};
    const double b[3] = {xk[0] - xj[0], xk[1] - xj[1], xk[2] - xj[2]};
    *ty = atan2(a[0] * b[1] - b[0] * a[1], a[0] * b[0] + a[1] * b[1]);
    *tz = atan2(a[0] * b[2] - b[0] * a[2], a[0] * b[0] + a[2] * b[2]);
}

// Forces of one bending spring on its three nodes (f[0..8] = F_i, F_j, F_k).
void bend_force(const Bend& s, const double* xi, const double* xj, const double* xk, double* f) {
    for (int q = 0; q < 9; ++q) f[q] = 0.0;
    const double a[3] = {xj[0] - xi[0], xj[1] - xi[1], xj[2] - xi[2]};
    const double b[3] = {xk[0] - xj[0], xk[1] - xj[1], xk[2] - xj[2]};
    // projected planes (x, y) and (x, z): the second component is q
    for (int q = 1; q <= 2; ++q) {
        const double A = a[0] * b[q] - b[0] * a[q], B = a[0] * b[0] + a[q] * b[q];
        const double r2 = A * A + B * B;
        if (r2 == 0.0) continue;
        // dtheta = (B dA - A dB) / r2; E = (1/2) k^b dth^2 -> dE = g (B dA - A dB)
        const double g = s.kb * wrap(atan2(A, B) - (q == 1 ? s.t0y : s.t0z)) / r2;
        // dA/da = (b_q, -b_0), dA/db = (-a_q, a_0); dB/da = (b_0, b_q), dB/db = (a_0, a_q)
        const double Ea0 = g * (B * b[q] - A * b[0]), Eaq = g * (-B * b[0] - A * b[q]);
        const double Eb0 = g * (-B * a[q] - A * a[0]), Ebq = g * (B * a[0] - A * a[q]);
        // a = x_j - x_i, b = x_k - x_j, F = -dE/dx
        f[0] += Ea0;
        f[q] += Eaq;
        f[3] += -Ea0 + Eb0;
        f[3 + q] += -Eaq + Ebq;
        f[6] += -Eb0;
        f[6 + q] += -Ebq;
    }
}

// Band matrix of order m, kl sub- and ku super-diagonals, with kl more
// super-diagonals for the fill of partial pivoting (column-major band).
struct Band {
    int m = 0, kl = 0, ku = 0, ld = 0;
    std::vector<double> ab;
    std::vector<int> piv;
    void reset(int m_, int kl_, int ku_) {
        m = m_;
        kl = kl_;
        ku = ku_;
        ld = 2 * kl + ku + 1;
        ab.assign((size_t)ld * m, 0.0);
        piv.assign(m, 0);
    }
    double& at(int i, int j) { return ab[(size_t)j * ld + (kl + ku + i - j)]; }
    void add(int i, int j, double v) { at(i, j) += v; }
    // LU with partial pivoting in place; false if a pivot is zero
    bool factor() {
        int ju = 0;
        for (int j = 0; j < m; ++j) {
            const int km = std::min(kl, m - 1 - j);
            int jp = 0;
            double best = fabs(at(j, j));
            for (int r = 1; r <= km; ++r)
                if (fabs(at(j + r, j)) > best) { best = fabs(at(j + r, j)); jp = r; }
            piv[j] = j + jp;
            if (best == 0.0) return false;
            ju = std::max(ju, std::min(j + ku + jp, m - 1));
            if (jp != 0)
                for (int c = j; c <= ju; ++c) std::swap(at(j, c), at(j + jp, c));
            const double inv = 1.0 / at(j, j);
            for (int r = 1; r <= km; ++r) at(j + r, j) *= inv;
            for (int c = j + 1; c <= ju; ++c) {
                const double u = at(j, c);
                if (u == 0.0) continue;
                for (int r = 1; r <= km; ++r) at(j + r, c) -= at(j + r, j) * u;
            }
        }
        return true;
    }
    void solve(double* b) {
        for (int j = 0; j < m; ++j) {
            if (piv[j] != j) std::swap(b[j], b[piv[j]]);
            const int km = std::min(kl, m - 1 - j);
            for (int r = 1; r <= km; ++r) b[j + r] -= at(j + r, j) * b[j];
        }
        for (int j = m - 1; j >= 0; --j) {
            b[j] /= at(j, j);
            const int i0 = std::max(0, j - kl - ku);
            for (int i = i0; i < j; ++i) b[i] -= at(i, j) * b[j];
        }
    }
};

double norm2(const std::vector<double>& a) {
    double s = 0.0;
    for (double q : a) s += q * q;
    return sqrt(s);
}

}  // namespace

struct ps_ms {
    int n = 0;
    std::vector<double> x, v, xm1, vm1, mass;
    std::vector<unsigned char> fixed;
    std::vector<Ext> ext;
    std::vector<Bend> bend;
    std::vector<int> pos;    // node -> place among the free nodes (RCM order), -1 if fixed
    int nfree = 0, bw = 0;   // free nodes, node bandwidth of the Newton matrix
    double dt_prev = 0.0;
    long steps = 0;
    Band J;
    bool j_valid = false;    // J holds a factored step matrix
    double j_cdt = 0.0;      // c dt it was built for
    long factorizations = 0;
    std::string err;

    // internal forces F = -grad E at positions y (3 n)
    void forces(const double* y, double* F) const {
        memset(F, 0, sizeof(double) * 3 * n);
        for (const Ext& e : ext) {
            double d[3], L = 0.0;
            for (int c = 0; c < 3; ++c) { d[c] = y[3 * e.j + c] - y[3 * e.i + c]; L += d[c] * d[c]; }
            L = sqrt(L);
            if (L == 0.0) continue;
            const double f = e.k * (L - e.l0) / L;   // along e_ij, on i
            for (int c = 0; c < 3; ++c) {
                F[3 * e.i + c] += f * d[c];
                F[3 * e.j + c] -= f * d[c];
            }
        }
        double f[9];
        for (const Bend& s : bend) {
            bend_force(s, y + 3 * s.i, y + 3 * s.j, y + 3 * s.k, f);
            const int nd[3] = {s.i, s.j, s.k};
            for (int t = 0; t < 3; ++t)
                for (int c = 0; c < 3; ++c) F[3 * nd[t] + c] += f[3 * t + c];
        }
    }

    // Reverse Cuthill--McKee order of the free nodes over the Newton
    // matrix's coupling graph (extension pairs, all pairs of a bending triple).
    void order() {
        std::vector<std::vector<int>> adj(n);
        auto link = [&](int a, int b) {
            if (a == b || fixed[a] || fixed[b]) return;
            adj[a].push_back(b);
            adj[b].push_back(a);
        };
        for (const Ext& e : ext) link(e.i, e.j);
        for (const Bend& s : bend) { link(s.i, s.j); link(s.j, s.k); link(s.i, s.k); }
        for (auto& a : adj) {
            std::sort(a.begin(), a.end());
            a.erase(std::unique(a.begin(), a.end()), a.end());
        }
        std::vector<int> seq;
        std::vector<char> seen(n, 0);
        for (;;) {
            int start = -1;
            for (int i = 0; i < n; ++i)
                if (!fixed[i] && !seen[i] && (start < 0 || adj[i].size() < adj[start].size())) start = i;
            if (start < 0) break;
            size_t head = seq.size();
            seq.push_back(start);
            seen[start] = 1;
            while (head < seq.size()) {
                const int u = seq[head++];
                std::vector<int> nb;
                for (int w : adj[u])
                    if (!seen[w]) { seen[w] = 1; nb.push_back(w); }
                std::sort(nb.begin(), nb.end(), [&](int p, int q) {
                    return adj[p].size() != adj[q].size() ? adj[p].size() < adj[q].size() : p < q;
                });
                seq.insert(seq.end(), nb.begin(), nb.end());
            }
        }
        std::reverse(seq.begin(), seq.end());
        pos.assign(n, -1);
        nfree = (int)seq.size();
        for (int p = 0; p < nfree; ++p) pos[seq[p]] = p;
        bw = 0;
        for (int i = 0; i < n; ++i)
            for (int w : adj[i]) bw = std::max(bw, abs(pos[i] - pos[w]));
    }

    void band_reset() { J.reset(3 * nfree, 3 * bw + 2, 3 * bw + 2); }

    // add dF/dx at positions y into J (free rows and columns only)
    void add_stiffness(const double* y) {
        for (const Ext& e : ext) {
            double d[3], L = 0.0;
            for (int c = 0; c < 3; ++c) { d[c] = y[3 * e.j + c] - y[3 * e.i + c]; L += d[c] * d[c]; }
            L = sqrt(L);
            if (L == 0.0) continue;
            // dF_i/dx_j = k [(1 - l0/L) I + (l0/L) e e^T] = -dF_i/dx_i
            double K[3][3];
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c)
                    K[r][c] = e.k * ((r == c ? 1.0 - e.l0 / L : 0.0) + e.l0 / L * d[r] * d[c] / (L * L));
            const int nd[2] = {e.i, e.j};
            for (int a = 0; a < 2; ++a) {
                if (pos[nd[a]] < 0) continue;
                for (int b = 0; b < 2; ++b) {
                    if (pos[nd[b]] < 0) continue;
                    const double sg = a == b ? -1.0 : 1.0;
                    for (int r = 0; r < 3; ++r)
                        for (int c = 0; c < 3; ++c) J.add(3 * pos[nd[a]] + r, 3 * pos[nd[b]] + c, sg * K[r][c]);
                }
            }
        }
        double loc[9], fp[9], fm[9];
        for (const Bend& sp : bend) {
            const int nd[3] = {sp.i, sp.j, sp.k};
            for (int t = 0; t < 3; ++t)
                for (int c = 0; c < 3; ++c) loc[3 * t + c] = y[3 * nd[t] + c];
            double scale = 0.0;
            for (int c = 0; c < 3; ++c)
                scale = fmax(scale, fmax(fabs(loc[3 + c] - loc[c]), fabs(loc[6 + c] - loc[3 + c])));
            const double h = 1e-6 * (scale > 0.0 ? scale : 1.0);
            for (int col = 0; col < 9; ++col) {
                const int pc = pos[nd[col / 3]];
                if (pc < 0) continue;
                const double keep = loc[col];
                loc[col] = keep + h;
                bend_force(sp, loc, loc + 3, loc + 6, fp);
                loc[col] = keep - h;
                bend_force(sp, loc, loc + 3, loc + 6, fm);
                loc[col] = keep;
                for (int row = 0; row < 9; ++row) {
                    const int pr = pos[nd[row / 3]];
                    if (pr < 0) continue;
                    J.add(3 * pr + row % 3, 3 * pc + col % 3, (fp[row] - fm[row]) / (2.0 * h));
                }
            }
        }
    }
};

extern "C" {

ps_status ps_ms_create(int32_t n_nodes, const double* mass, const double* x0, const double* v0,
                       const unsigned char* fixed, int32_t n_ext, const int32_t* ext_ij, const double* ke,
                       int32_t n_bend, const int32_t* bend_ijk, const double* kb, ps_ms** out) {
    if (!out) return PS_EINVAL;
    *out = nullptr;
    if (n_nodes < 1 || !mass || !x0 || n_ext < 0 || n_bend < 0 || (n_ext > 0 && (!ext_ij || !ke)) ||
        (n_bend > 0 && (!bend_ijk || !kb)))
        return PS_EINVAL;
    for (int i = 0; i < n_nodes; ++i)
        if (!(mass[i] > 0.0)) return PS_EINVAL;
    for (int s = 0; s < n_ext; ++s) {
        const int i = ext_ij[2 * s], j = ext_ij[2 * s + 1];
        if (i < 0 || i >= n_nodes || j < 0 || j >= n_nodes || i == j) return PS_EINVAL;
    }
    for (int s = 0; s < n_bend; ++s) {
        const int i = bend_ijk[3 * s], j = bend_ijk[3 * s + 1], k = bend_ijk[3 * s + 2];
        if (i < 0 || i >= n_nodes || j < 0 || j >= n_nodes || k < 0 || k >= n_nodes || i == j || j == k || i == k)
            return PS_EINVAL;
    }
    ps_ms* m = ps_fault_alloc("ms") ? nullptr : new (std::nothrow) ps_ms();
    if (!m) return PS_ENOMEM;
    m->n = n_nodes;
    m->x.assign(x0, x0 + 3 * n_nodes);
    m->v.assign(3 * n_nodes, 0.0);
    if (v0) m->v.assign(v0, v0 + 3 * n_nodes);
    m->mass.assign(mass, mass + n_nodes);
    m->fixed.assign(n_nodes, 0);
    if (fixed)
        for (int i = 0; i < n_nodes; ++i) m->fixed[i] = fixed[i] ? 1 : 0;
    for (int i = 0; i < n_nodes; ++i)
        if (m->fixed[i])
            for (int c = 0; c < 3; ++c) m->v[3 * i + c] = 0.0;
    for (int s = 0; s < n_ext; ++s) {
        Ext e;
        e.i = ext_ij[2 * s];
        e.j = ext_ij[2 * s + 1];
        e.k = ke[s];
        double L = 0.0;
        for (int c = 0; c < 3; ++c) L += (x0[3 * e.j + c] - x0[3 * e.i + c]) * (x0[3 * e.j + c] - x0[3 * e.i + c]);
        e.l0 = sqrt(L);
        m->ext.push_back(e);
    }
    for (int s = 0; s < n_bend; ++s) {
        Bend b;
        b.i = bend_ijk[3 * s];
        b.j = bend_ijk[3 * s + 1];
        b.k = bend_ijk[3 * s + 2];
        b.kb = kb[s];
        bend_angles(x0 + 3 * b.i, x0 + 3 * b.j, x0 + 3 * b.k, &b.t0y, &b.t0z);
        m->bend.push_back(b);
    }
    m->order();
    *out = m;
    return PS_OK;
}

ps_status ps_ms_destroy(ps_ms* m) {
    delete m;
    return PS_OK;
}

ps_status ps_ms_info(const ps_ms* m, int32_t* n_free, int32_t* bandwidth, int64_t* factorizations) {
    if (!m) return PS_EINVAL;
    if (n_free) *n_free = m->nfree;
    if (bandwidth) *bandwidth = m->bw;
    if (factorizations) *factorizations = m->factorizations;
    return PS_OK;
}

ps_status ps_ms_forces(const ps_ms* m, const double* x, double* f_out) {
    if (!m || !x || !f_out) return PS_EINVAL;
    m->forces(x, f_out);
    return PS_OK;
}

ps_status ps_ms_state(const ps_ms* m, double* x_out, double* v_out) {
    if (!m) return PS_EINVAL;
    if (x_out) memcpy(x_out, m->x.data(), sizeof(double) * 3 * m->n);
    if (v_out) memcpy(v_out, m->v.data(), sizeof(double) * 3 * m->n);
    return PS_OK;
}

ps_status ps_ms_set_state(ps_ms* m, const double* x, const double* v) {
    if (!m || !x) return PS_EINVAL;
    m->x.assign(x, x + 3 * m->n);
    if (v) m->v.assign(v, v + 3 * m->n);
    else m->v.assign(3 * m->n, 0.0);
    for (int i = 0; i < m->n; ++i)
        if (m->fixed[i])
            for (int c = 0; c < 3; ++c) m->v[3 * i + c] = 0.0;
    m->steps = 0;
    m->j_valid = false;
    return PS_OK;
}

ps_status ps_ms_step(ps_ms* m, double dt, const double* f_ext, const ps_ms_frame* frame, double tol,
                     int32_t max_iter, int32_t* iters_out) {
    if (!m || !(dt > 0.0) || !(tol > 0.0) || max_iter < 1) return PS_EINVAL;
    const int n = m->n, n3 = 3 * n;
    const double xi = m->steps == 0 ? 0.0 : dt / m->dt_prev;
    const double a = (1 + xi) * (1 + xi) / (1 + 2 * xi), b = xi * xi / (1 + 2 * xi), c = (1 + xi) / (1 + 2 * xi);
    const double cdt = c * dt;
    const std::vector<double>& xm1 = m->steps == 0 ? m->x : m->xm1;
    const std::vector<double>& vm1 = m->steps == 0 ? m->v : m->vm1;
    std::vector<double> hx(n3), hv(n3);
    for (int q = 0; q < n3; ++q) {
        hx[q] = a * m->x[q] - b * xm1[q];
        hv[q] = a * m->v[q] - b * vm1[q];
    }
    // frame terms: f = -m (A_O + G y + 2 W v), G = [dOmega]x + [Omega]x [Omega]x, W = [Omega]x
    double W[3][3] = {}, G[3][3] = {}, A0[3] = {0.0, 0.0, 0.0};
    if (frame) {
        const double* w = frame->Omega;
        const double* dw = frame->dOmega;
        const double Wm[3][3] = {{0, -w[2], w[1]}, {w[2], 0, -w[0]}, {-w[1], w[0], 0}};
        const double Dm[3][3] = {{0, -dw[2], dw[1]}, {dw[2], 0, -dw[0]}, {-dw[1], dw[0], 0}};
        for (int r = 0; r < 3; ++r) {
            A0[r] = frame->A_O[r];
            for (int q = 0; q < 3; ++q) {
                W[r][q] = Wm[r][q];
                G[r][q] = Dm[r][q];
                for (int t = 0; t < 3; ++t) G[r][q] += Wm[r][t] * Wm[t][q];
            }
        }
    }
    const int mf = 3 * m->nfree;
    std::vector<double> y(m->x), F(n3), r(mf);
    // Newton matrix I/cdt - (cdt/m) dF/dy + cdt G + 2 W at y, factored
    auto build = [&]() -> bool {
        m->band_reset();
        m->add_stiffness(y.data());
        Band& Jb = m->J;
        for (int i = 0; i < n; ++i) {
            const int p = m->pos[i];
            if (p < 0) continue;
            const double s = -cdt / m->mass[i];
            for (int q = 0; q < 3; ++q) {
                const int row = 3 * p + q;
                const int c0 = std::max(0, row - Jb.kl), c1 = std::min(Jb.m - 1, row + Jb.ku);
                for (int col = c0; col <= c1; ++col) Jb.at(row, col) *= s;
                Jb.at(row, row) += 1.0 / cdt;
                if (frame)
                    for (int t = 0; t < 3; ++t) Jb.add(row, 3 * p + t, cdt * G[q][t] + 2.0 * W[q][t]);
            }
        }
        m->factorizations++;
        m->j_cdt = cdt;
        m->j_valid = Jb.factor();
        return m->j_valid;
    };
    // Simplified Newton: the factored matrix of an earlier iteration or step
    // is reused while the iteration contracts fast (rate <= 1/2, at most six
    // iterations); otherwise, or when c dt changed by more than 20 %, it is
    // rebuilt at the current iterate and the iteration goes on from there. Converged when the
    // update, scaled by rate/(1 - rate) once a rate is known (the remaining
    // error of a linearly converging iteration), is below tol * max(1, |y|).
    bool fresh = false;
    if (!m->j_valid || fabs(cdt / m->j_cdt - 1.0) > 0.2) {
        if (!build()) {
            m->err = "ps_ms_step: singular Newton matrix";
            return PS_ENUMERIC;
        }
        fresh = true;
    }
    int it = 0;
    bool conv = false;
    double dn_prev = -1.0;
    for (it = 1; it <= max_iter; ++it) {
        // residual of the velocity equation with v = (y - hx)/cdt, on free coordinates
        m->forces(y.data(), F.data());
        for (int i = 0; i < n; ++i) {
            const int p = m->pos[i];
            if (p < 0) continue;
            double vy[3];
            for (int q = 0; q < 3; ++q) vy[q] = (y[3 * i + q] - hx[3 * i + q]) / cdt;
            for (int q = 0; q < 3; ++q) {
                double fi = F[3 * i + q] + (f_ext ? f_ext[3 * i + q] : 0.0);
                if (frame) {
                    double g = A0[q];
                    for (int t = 0; t < 3; ++t) g += G[q][t] * y[3 * i + t] + 2.0 * W[q][t] * vy[t];
                    fi -= m->mass[i] * g;
                }
                r[3 * p + q] = -(vy[q] - hv[3 * i + q] - cdt * fi / m->mass[i]);
            }
        }
        m->J.solve(r.data());
        const double dn = norm2(r);
        if (!(dn == dn)) break;
        const double rate = dn_prev > 0.0 ? dn / dn_prev : -1.0;
        if (!fresh && (rate > 0.5 || it > 6)) {
            // too slow with the old matrix: rebuild at y and take this iteration again
            if (!build()) {
                m->err = "ps_ms_step: singular Newton matrix";
                return PS_ENUMERIC;
            }
            fresh = true;
            dn_prev = -1.0;
            continue;
        }
        if (rate >= 1.0) break;   // diverging even with a fresh matrix
        double yn = 0.0;
        for (int i = 0; i < n; ++i) {
            const int p = m->pos[i];
            if (p < 0) continue;
            for (int q = 0; q < 3; ++q) {
                y[3 * i + q] += r[3 * p + q];
                yn += y[3 * i + q] * y[3 * i + q];
            }
        }
        const double est = rate > 0.0 ? dn * rate / (1.0 - rate) : dn;
        if (est < tol * fmax(1.0, sqrt(yn)) && (rate > 0.0 || fresh)) {
            conv = true;
            break;
        }
        dn_prev = dn;
    }
    if (iters_out) *iters_out = conv ? it : max_iter;
    if (!conv) {
        m->err = "ps_ms_step: Newton did not converge";
        return PS_ENUMERIC;
    }
    m->xm1 = m->x;
    m->vm1 = m->v;
    for (int q = 0; q < n3; ++q) m->v[q] = m->fixed[q / 3] ? 0.0 : (y[q] - hx[q]) / cdt;
    m->x = y;
    m->dt_prev = dt;
    m->steps++;
    return PS_OK;
}

ps_status ps_ms_equilibrium(ps_ms* m, const double* f_ext, int32_t load_steps, double tol, int32_t max_iter,
                            int32_t* iters_out) {
    if (!m || !f_ext || load_steps < 1 || !(tol > 0.0) || max_iter < 1) return PS_EINVAL;
    const int n = m->n, n3 = 3 * n, mf = 3 * m->nfree;
    std::vector<double> F(n3), r(mf), x(m->x);
    int total = 0;
    for (int s = 1; s <= load_steps; ++s) {
        const double w = (double)s / load_steps;
        bool conv = false;
        for (int it = 0; it < max_iter; ++it) {
            ++total;
            m->forces(x.data(), F.data());
            for (int i = 0; i < n; ++i) {
                const int p = m->pos[i];
                if (p < 0) continue;
                for (int q = 0; q < 3; ++q) r[3 * p + q] = -(F[3 * i + q] + w * f_ext[3 * i + q]);
            }
            m->band_reset();
            m->add_stiffness(x.data());
            m->factorizations++;
            if (!m->J.factor()) {
                m->err = "ps_ms_equilibrium: singular stiffness";
                if (iters_out) *iters_out = total;
                return PS_ENUMERIC;
            }
            m->J.solve(r.data());
            double xn = 0.0;
            for (int i = 0; i < n; ++i) {
                const int p = m->pos[i];
                if (p < 0) continue;
                for (int q = 0; q < 3; ++q) {
                    x[3 * i + q] += r[3 * p + q];
                    xn += x[3 * i + q] * x[3 * i + q];
                }
            }
            const double dn = norm2(r);
            if (!(dn == dn)) break;
            if (dn < tol * fmax(1.0, sqrt(xn))) {
                conv = true;
                break;
            }
        }
        if (!conv) {
            m->err = "ps_ms_equilibrium: Newton did not converge";
            if (iters_out) *iters_out = total;
            return PS_ENUMERIC;
        }
    }
    m->x = x;
    m->v.assign(n3, 0.0);
    m->steps = 0;
    m->j_valid = false;
    if (iters_out) *iters_out = total;
    return PS_OK;
}

// Checkpoint layout: 8-byte tag, node count, step count (int64), previous
// step (double), then x, v, x^{n-1}, v^{n-1} (3n doubles each).
static const char kMsTag[8] = {'p', 's', 'm', 's', 'v', '0', '0', '1'};

ps_status ps_ms_state_size(const ps_ms* m, size_t* bytes) {
    if (!m || !bytes) return PS_EINVAL;
    *bytes = 32 + 4 * sizeof(double) * 3 * (size_t)m->n;
    return PS_OK;
}

ps_status ps_ms_save(ps_ms* m, void* buf) {
    if (!m || !buf) return PS_EINVAL;
    unsigned char* d = (unsigned char*)buf;
    const int64_t hdr[2] = {m->n, m->steps};
    memcpy(d, kMsTag, 8);
    memcpy(d + 8, hdr, 16);
    memcpy(d + 24, &m->dt_prev, 8);
    const size_t b = sizeof(double) * 3 * (size_t)m->n;
    memcpy(d + 32, m->x.data(), b);
    memcpy(d + 32 + b, m->v.data(), b);
    const bool hist = m->steps > 0;
    memcpy(d + 32 + 2 * b, (hist ? m->xm1 : m->x).data(), b);
    memcpy(d + 32 + 3 * b, (hist ? m->vm1 : m->v).data(), b);
    // the next step rebuilds its Newton matrix, as a restored network does
    m->j_valid = false;
    return PS_OK;
}

ps_status ps_ms_restore(ps_ms* m, const void* buf) {
    if (!m || !buf) return PS_EINVAL;
    const unsigned char* d = (const unsigned char*)buf;
    int64_t hdr[2];
    memcpy(hdr, d + 8, 16);
    if (memcmp(d, kMsTag, 8) != 0 || hdr[0] != m->n || hdr[1] < 0) {
        m->err = "ps_ms_restore: not a state of a network with this node count";
        return PS_EINVAL;
    }
    const double* q = (const double*)(d + 32);
    const size_t n3 = 3 * (size_t)m->n;
    memcpy(&m->dt_prev, d + 24, 8);
    m->steps = (long)hdr[1];
    m->x.assign(q, q + n3);
    m->v.assign(q + n3, q + 2 * n3);
    m->xm1.assign(q + 2 * n3, q + 3 * n3);
    m->vm1.assign(q + 3 * n3, q + 4 * n3);
    m->j_valid = false;
    return PS_OK;
}

const char* ps_ms_last_error(const ps_ms* m) { return m ? m->err.c_str() : ""; }

}  // extern "C"
