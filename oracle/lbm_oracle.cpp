// ORACLE — test infrastructure only.
//
// Plain, slow, FP64 CPU implementation of the two-component Shan-Chen
// lattice Boltzmann step with exact-flow ghost boundaries, written from the
// paper's equations (Milan, Biferale, Sbragaglia, Toschi, "Sub-Kolmogorov
// droplet dynamics in isotropic turbulence using a multiscale Lattice
// Boltzmann scheme", Sec. 2 Eqs. 6-10 and Sec. 3 Eq. 14).  Only tests/,
// __graft_entry__.smoke() and bench.py's CPU-baseline leg may load it.  It
// shares no code, table or helper with the CUDA library.
//
// Every step is taken in the order the method states it, with no blocking,
// fusion or reordering:
//   (i)   ghost populations g_i^eq(rho_b, A(t) x) on the one-layer shell
//         outside the box (Sec. 2, Eq. 8; Sec. 3, Eq. 14),
//   (ii)  pull streaming g_i(x, t+1) = g*_i(x - c_i, t) (Eq. 9),
//   (iii) component densities rho_sigma = sum_i g_i^sigma (Eq. 6),
//   (iv)  Shan-Chen force F^sigma = -G rho_sigma sum_i w_i rho_sigma'(x+c_i) c_i
//         (Eq. 7; out-of-box neighbours take the ghost density rho_b),
//   (v)   common velocity u' = sum_s j_s/tau_s / sum_s rho_s/tau_s and the
//         shifted equilibrium velocity u_s = u' + tau_s F^s / rho_s
//         (Shan-Chen forcing, the model of Sec. 2),
//   (vi)  BGK relaxation g* = g - (g - g^eq(rho_s, u_s)) / tau_s with
//         nu = (tau - 1/2)/3 (Eqs. 9, 10).
//
// Optional storage model (orc_set_storage): after every state change the
// populations are replaced by the values that 16-bit deviation storage can
// hold, so the same oracle states what that storage form of the method
// computes.  A population streaming from x to x + c_i is kept as the
// deviation d_i = f*_i - w_i rho*(x + c_i), rounded to binary16 or bfloat16,
// with rho* the float32 density of the node it streams to (the ghost density
// outside the box); the rest population holds the remainder of the node's
// float32 density, rounded to float32.  Ghost populations are held the same
// way, relative to the density of the fluid node they stream into.  This is
// an addition of the library, not of the paper: the paper stores populations
// at full precision.
//
// Optional MRT collision (orc_set_mrt), the multi-relaxation-time operator
// Sec. 2 names: g* = g - M^-1 S M (g - g^eq), M the D3Q19 moment basis of
// d'Humieres et al. (2002) (orthogonal rows, polynomials in c: density,
// energy, energy square, momentum, energy flux, stress and its
// higher-order partners, third-order moments), S = diag of the relaxation
// rates.  The stress moments relax at 1/tau_s (Eq. 10); the momentum moments
// also at 1/tau_s, so that the velocity shift of the forcing still puts F^s
// into the fluid; the other rates are parameters.  With every rate 1/tau_s it
// is the BGK operator.
//
// Build: g++ -O2 -ffp-contract=off -fopenmp -shared -fPIC (see build.py).
// Loops over nodes run in parallel over the rows (z, y) of boxes of at
// least 32768 nodes; smaller boxes run on one thread, where starting the
// threads would cost more than the work.  Every node's result is
// independent of the thread count.  The moment and checksum sums are serial
// and ordered z, y, x.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// Whether a loop over the nodes of an Lx x Ly x Lz box is worth threads.
bool parallel_worth(int Lx, int Ly, int Lz) { return (long long)Ly * Lz > 1 && (long long)Lx * Ly * Lz >= 32768; }

// D3Q19 velocity set, in the order used throughout this repository:
// rest, the six axis vectors (+x,-x,+y,-y,+z,-z), then the twelve
// face diagonals, each followed by its opposite.
const int CX[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
const int CY[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
const int CZ[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

double weight(int i) {
    if (i == 0) return 1.0 / 3.0;
    if (i <= 6) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

// Eq. 8: g_i^eq = rho w_i (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u)
double equilibrium(int i, double rho, const double u[3]) {
    double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return rho * weight(i) * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

// Row k of the D3Q19 moment basis of d'Humieres et al. (2002) at velocity c:
// 0 rho, 1 e, 2 eps, 3 j_x, 4 q_x, 5 j_y, 6 q_y, 7 j_z, 8 q_z, 9 3p_xx,
// 10 3pi_xx, 11 p_ww, 12 pi_ww, 13 p_xy, 14 p_yz, 15 p_xz, 16 m_x, 17 m_y, 18 m_z.
double moment_row(int k, int cx, int cy, int cz) {
    const double c2 = cx * cx + cy * cy + cz * cz;
    switch (k) {
        case 0: return 1.0;
        case 1: return 19.0 * c2 - 30.0;
        case 2: return (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0;
        case 3: return cx;
        case 4: return (5.0 * c2 - 9.0) * cx;
        case 5: return cy;
        case 6: return (5.0 * c2 - 9.0) * cy;
        case 7: return cz;
        case 8: return (5.0 * c2 - 9.0) * cz;
        case 9: return 3.0 * cx * cx - c2;
        case 10: return (3.0 * c2 - 5.0) * (3.0 * cx * cx - c2);
        case 11: return cy * cy - cz * cz;
        case 12: return (3.0 * c2 - 5.0) * (cy * cy - cz * cz);
        case 13: return cx * cy;
        case 14: return cy * cz;
        case 15: return cx * cz;
        case 16: return (cy * cy - cz * cz) * cx;
        case 17: return (cz * cz - cx * cx) * cy;
        default: return (cx * cx - cy * cy) * cz;
    }
}

// Relaxation rate of moment k for component relaxation time tau.
double moment_rate(int k, double tau, const double* r) {
    if (k == 0 || k == 3 || k == 5 || k == 7) return 1.0 / tau;  // density (any rate) and momentum
    if (k == 9 || k == 11 || k == 13 || k == 14 || k == 15) return 1.0 / tau;  // stress: viscosity, Eq. 10
    if (k == 1) return r[0];
    if (k == 2) return r[1];
    if (k == 4 || k == 6 || k == 8) return r[2];
    if (k == 10 || k == 12) return r[3];
    return r[4];  // 16, 17, 18
}

// x rounded to nearest-even in a binary format with p significant bits and
// smallest normal exponent emin (gradual underflow below it); the values
// rounded here are far below every format's largest finite number.
double round_to_format(double x, int p, int emin) {
    if (x == 0.0 || !std::isfinite(x)) return x;
    int e;
    std::frexp(x, &e);  // |x| = m 2^e, 1/2 <= m < 1: leading bit 2^(e-1)
    int lead = e - 1;
    if (lead < emin) lead = emin;
    const double q = std::ldexp(1.0, lead - (p - 1));  // spacing of the format near x
    return std::nearbyint(x / q) * q;                   // default mode: ties to even
}
double to_float32(double x) { return round_to_format(x, 24, -126); }
double to_binary16(double x) { return round_to_format(x, 11, -14); }
double to_bfloat16(double x) { return round_to_format(x, 8, -126); }

struct Oracle {
    int L[3];
    bool periodic;
    int storage = 0;  // 0 full precision, 1 binary16 deviations, 2 bfloat16 deviations
    bool mrt = false;
    double mrt_rates[5] = {0, 0, 0, 0, 0};  // s_e, s_eps, s_q, s_pi, s_m
    double tau[2];
    double G;
    double rho_b[2];
    std::vector<double> fpost;   // post-collision populations [2][19][z][y][x]
    std::vector<double> fstream; // post-streaming populations, same layout
    std::vector<double> rho;     // [2][z][y][x]

    int64_t nodes() const { return (int64_t)L[0] * L[1] * L[2]; }
    int64_t node(int x, int y, int z) const { return ((int64_t)z * L[1] + y) * L[0] + x; }
    int64_t pidx(int s, int i, int64_t n) const { return ((int64_t)s * 19 + i) * nodes() + n; }
    bool inside(int x, int y, int z) const {
        return x >= 0 && x < L[0] && y >= 0 && y < L[1] && z >= 0 && z < L[2];
    }
    // Coordinates are measured from the box centre, where the droplet's
    // centre of mass sits (Sec. 3, Eq. 14).
    void position(int x, int y, int z, double p[3]) const {
        p[0] = x - 0.5 * (L[0] - 1);
        p[1] = y - 0.5 * (L[1] - 1);
        p[2] = z - 0.5 * (L[2] - 1);
    }
    static int wrap(int a, int n) { return ((a % n) + n) % n; }

    // Density of component s at (x, y, z) after streaming; nodes outside the
    // box carry the ghost density rho_b (or the periodic image).
    double density_at(int s, int x, int y, int z) const {
        if (periodic) {
            x = wrap(x, L[0]); y = wrap(y, L[1]); z = wrap(z, L[2]);
        } else if (!inside(x, y, z)) {
            return rho_b[s];
        }
        return rho[(int64_t)s * nodes() + node(x, y, z)];
    }

    // The storage model: replace fpost by what 16-bit deviation storage holds.
    void apply_storage() {
        if (storage == 0) return;
        const int64_t N = nodes();
        // float32 densities of the stored state (the rest of the state refers to them)
        std::vector<double> rs((size_t)(2 * N));
        for (int s = 0; s < 2; ++s)
            for (int64_t n = 0; n < N; ++n) {
                double r = 0.0;
                for (int i = 0; i < 19; ++i) r += fpost[pidx(s, i, n)];
                rs[(size_t)(s * N + n)] = to_float32(r);
            }
        auto dest = [&](int s, int x, int y, int z) {
            if (periodic) {
                x = wrap(x, L[0]); y = wrap(y, L[1]); z = wrap(z, L[2]);
            } else if (!inside(x, y, z)) {
                return to_float32(rho_b[s]);
            }
            return rs[(size_t)(s * N + node(x, y, z))];
        };
#pragma omp parallel for collapse(2) schedule(static) if (parallel_worth(L[0], L[1], L[2]))
        for (int z = 0; z < L[2]; ++z)
            for (int y = 0; y < L[1]; ++y)
                for (int x = 0; x < L[0]; ++x) {
                    const int64_t n = node(x, y, z);
                    for (int s = 0; s < 2; ++s) {
                        double moving = 0.0;
                        for (int i = 1; i < 19; ++i) {
                            const double ref = weight(i) * dest(s, x + CX[i], y + CY[i], z + CZ[i]);
                            const double d = fpost[pidx(s, i, n)] - ref;
                            const double dq = storage == 1 ? to_binary16(d) : to_bfloat16(d);
                            fpost[pidx(s, i, n)] = ref + dq;
                            moving += ref + dq;
                        }
                        fpost[pidx(s, 0, n)] = to_float32(rs[(size_t)(s * N + n)] - moving);
                    }
                }
    }
};

}  // namespace

extern "C" {

void* orc_create(int Lx, int Ly, int Lz, int periodic, double tau_a, double tau_b, double G,
                 double rho_b_a, double rho_b_b) {
    Oracle* o = new Oracle();
    o->L[0] = Lx; o->L[1] = Ly; o->L[2] = Lz;
    o->periodic = periodic != 0;
    o->tau[0] = tau_a; o->tau[1] = tau_b;
    o->G = G;
    o->rho_b[0] = rho_b_a; o->rho_b[1] = rho_b_b;
    o->fpost.assign((size_t)(2 * 19 * o->nodes()), 0.0);
    o->fstream.assign((size_t)(2 * 19 * o->nodes()), 0.0);
    o->rho.assign((size_t)(2 * o->nodes()), 0.0);
    return o;
}

void orc_destroy(void* h) { delete (Oracle*)h; }

void orc_set_populations(void* h, const double* f) {
    Oracle* o = (Oracle*)h;
    std::memcpy(o->fpost.data(), f, o->fpost.size() * sizeof(double));
    o->apply_storage();
}

// Storage model: 0 full precision (the default), 1 binary16 deviations,
// 2 bfloat16 deviations.  Applies to the current state at once.  Returns 0,
// or -1 for an unknown mode.
int orc_set_storage(void* h, int mode) {
    Oracle* o = (Oracle*)h;
    if (mode < 0 || mode > 2) return -1;
    o->storage = mode;
    o->apply_storage();
    return 0;
}

// MRT collision: enable != 0 with rates[5] = {s_e, s_eps, s_q, s_pi, s_m};
// enable == 0 returns to BGK.
void orc_set_mrt(void* h, int enable, const double* rates) {
    Oracle* o = (Oracle*)h;
    o->mrt = enable != 0;
    if (rates)
        for (int k = 0; k < 5; ++k) o->mrt_rates[k] = rates[k];
}

// The moment basis, exported for its tests: M[19][19], M[k][i] = row k at c_i.
void orc_moment_basis(double* M) {
    for (int k = 0; k < 19; ++k)
        for (int i = 0; i < 19; ++i) M[19 * k + i] = moment_row(k, CX[i], CY[i], CZ[i]);
}

// The rounding of the storage model, exported for its tests:
// format 0 float32, 1 binary16, 2 bfloat16.
double orc_round(int format, double x) {
    if (format == 0) return to_float32(x);
    if (format == 1) return to_binary16(x);
    return to_bfloat16(x);
}

void orc_get_populations(void* h, double* f) {
    Oracle* o = (Oracle*)h;
    std::memcpy(f, o->fpost.data(), o->fpost.size() * sizeof(double));
}

// Initial state: component A (the droplet) follows a tanh profile of width
// xi around radius R, component B its complement; every population starts at
// the equilibrium of its local density and the linear flow u0 = A0 x.
void orc_init_droplet(void* h, double R, double xi, double rho_hi, double rho_lo, const double* A0) {
    Oracle* o = (Oracle*)h;
    for (int z = 0; z < o->L[2]; ++z)
        for (int y = 0; y < o->L[1]; ++y)
            for (int x = 0; x < o->L[0]; ++x) {
                double p[3];
                o->position(x, y, z, p);
                double r = std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
                double th = std::tanh((r - R) / xi);
                double rho_s[2];
                rho_s[0] = rho_lo + (rho_hi - rho_lo) * 0.5 * (1.0 - th);
                rho_s[1] = rho_lo + (rho_hi - rho_lo) * 0.5 * (1.0 + th);
                double u[3];
                for (int a = 0; a < 3; ++a)
                    u[a] = A0[3 * a + 0] * p[0] + A0[3 * a + 1] * p[1] + A0[3 * a + 2] * p[2];
                int64_t n = o->node(x, y, z);
                for (int s = 0; s < 2; ++s)
                    for (int i = 0; i < 19; ++i) o->fpost[o->pidx(s, i, n)] = equilibrium(i, rho_s[s], u);
            }
    o->apply_storage();
}

// One time step with the boundary gradient A (row-major, A[3*a+b] = d_b u_a).
// The ghost flow is u = A (x - x_c): linear in the distance from the frame
// origin x_c (Sec. 3, Eq. 14), which is the droplet's centre of mass when
// `centre` is given and the box centre when it is NULL.
// If flux_in / flux_out are given, they receive per component the mass that
// streamed in from ghost nodes and the post-collision mass that streamed out
// of the box during this step (exact bookkeeping of the open boundary).
void orc_step(void* h, const double* A, const double* centre, double* flux_in, double* flux_out) {
    Oracle* o = (Oracle*)h;
    const int Lx = o->L[0], Ly = o->L[1], Lz = o->L[2];
    const int64_t N = o->nodes();

    // Storage model: ghost populations are held in the same format as the
    // state, as deviations from w_i rho* of the fluid node they stream into.
    std::vector<double> rs;
    if (o->storage) {
        rs.resize((size_t)(2 * N));
        for (int s = 0; s < 2; ++s)
            for (int64_t n = 0; n < N; ++n) {
                double r = 0.0;
                for (int i = 0; i < 19; ++i) r += o->fpost[o->pidx(s, i, n)];
                rs[(size_t)(s * N + n)] = to_float32(r);
            }
    }

    // (i)+(ii) pull streaming, with ghost equilibria outside the box.
#pragma omp parallel for collapse(2) schedule(static) if (parallel_worth(Lx, Ly, Lz))
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < Ly; ++y)
            for (int x = 0; x < Lx; ++x) {
                int64_t n = o->node(x, y, z);
                for (int s = 0; s < 2; ++s)
                    for (int i = 0; i < 19; ++i) {
                        int xs = x - CX[i], ys = y - CY[i], zs = z - CZ[i];
                        double val;
                        if (o->periodic) {
                            int64_t m = o->node(Oracle::wrap(xs, Lx), Oracle::wrap(ys, Ly), Oracle::wrap(zs, Lz));
                            val = o->fpost[o->pidx(s, i, m)];
                        } else if (o->inside(xs, ys, zs)) {
                            val = o->fpost[o->pidx(s, i, o->node(xs, ys, zs))];
                        } else {
                            double p[3], u[3];
                            o->position(xs, ys, zs, p);
                            if (centre)
                                for (int a = 0; a < 3; ++a) p[a] -= centre[a];
                            for (int a = 0; a < 3; ++a)
                                u[a] = A[3 * a + 0] * p[0] + A[3 * a + 1] * p[1] + A[3 * a + 2] * p[2];
                            val = equilibrium(i, o->rho_b[s], u);
                            if (o->storage) {
                                const double ref = weight(i) * rs[(size_t)(s * N + n)];
                                const double d = val - ref;
                                val = ref + (o->storage == 1 ? to_binary16(d) : to_bfloat16(d));
                            }
                        }
                        o->fstream[o->pidx(s, i, n)] = val;
                    }
            }

    if (flux_in && flux_out) {
        for (int s = 0; s < 2; ++s) {
            double fin = 0.0, fout = 0.0;
            for (int z = 0; z < Lz; ++z)
                for (int y = 0; y < Ly; ++y)
                    for (int x = 0; x < Lx; ++x) {
                        int64_t n = o->node(x, y, z);
                        for (int i = 0; i < 19; ++i) {
                            if (o->periodic) continue;
                            if (!o->inside(x - CX[i], y - CY[i], z - CZ[i])) fin += o->fstream[o->pidx(s, i, n)];
                            if (!o->inside(x + CX[i], y + CY[i], z + CZ[i])) fout += o->fpost[o->pidx(s, i, n)];
                        }
                    }
            flux_in[s] = fin;
            flux_out[s] = fout;
        }
    }

    // (iii) densities after streaming.
#pragma omp parallel for collapse(2) schedule(static) if (parallel_worth(Lx, Ly, Lz))
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < Ly; ++y)
            for (int x = 0; x < Lx; ++x) {
                int64_t n = o->node(x, y, z);
                for (int s = 0; s < 2; ++s) {
                    double r = 0.0;
                    for (int i = 0; i < 19; ++i) r += o->fstream[o->pidx(s, i, n)];
                    o->rho[(int64_t)s * N + n] = r;
                }
            }

    // (iv)-(vi) force, velocities, collision.
#pragma omp parallel for collapse(2) schedule(static) if (parallel_worth(Lx, Ly, Lz))
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < Ly; ++y)
            for (int x = 0; x < Lx; ++x) {
                int64_t n = o->node(x, y, z);
                double rho_s[2], j[2][3], F[2][3];
                for (int s = 0; s < 2; ++s) {
                    rho_s[s] = o->rho[(int64_t)s * N + n];
                    j[s][0] = j[s][1] = j[s][2] = 0.0;
                    for (int i = 0; i < 19; ++i) {
                        double f = o->fstream[o->pidx(s, i, n)];
                        j[s][0] += f * CX[i];
                        j[s][1] += f * CY[i];
                        j[s][2] += f * CZ[i];
                    }
                }
                for (int s = 0; s < 2; ++s) {
                    int sp = 1 - s;  // the other component (G_AA = G_BB = 0)
                    double acc[3] = {0.0, 0.0, 0.0};
                    for (int i = 1; i < 19; ++i) {
                        double r = o->density_at(sp, x + CX[i], y + CY[i], z + CZ[i]);
                        acc[0] += weight(i) * r * CX[i];
                        acc[1] += weight(i) * r * CY[i];
                        acc[2] += weight(i) * r * CZ[i];
                    }
                    for (int a = 0; a < 3; ++a) F[s][a] = -o->G * rho_s[s] * acc[a];
                }
                double den = rho_s[0] / o->tau[0] + rho_s[1] / o->tau[1];
                double ucommon[3];
                for (int a = 0; a < 3; ++a) ucommon[a] = (j[0][a] / o->tau[0] + j[1][a] / o->tau[1]) / den;
                for (int s = 0; s < 2; ++s) {
                    double ueq[3];
                    for (int a = 0; a < 3; ++a) ueq[a] = ucommon[a] + o->tau[s] * F[s][a] / rho_s[s];
                    if (!o->mrt) {
                        for (int i = 0; i < 19; ++i) {
                            double f = o->fstream[o->pidx(s, i, n)];
                            double geq = equilibrium(i, rho_s[s], ueq);
                            o->fpost[o->pidx(s, i, n)] = f - (f - geq) / o->tau[s];
                        }
                    } else {
                        // g* = g - M^T D^-1 S M (g - g_eq), D = diag of the row norms
                        double dev[19], rel[19];
                        for (int i = 0; i < 19; ++i)
                            dev[i] = o->fstream[o->pidx(s, i, n)] - equilibrium(i, rho_s[s], ueq);
                        for (int k = 0; k < 19; ++k) {
                            double mk = 0.0, norm = 0.0;
                            for (int i = 0; i < 19; ++i) {
                                const double e = moment_row(k, CX[i], CY[i], CZ[i]);
                                mk += e * dev[i];
                                norm += e * e;
                            }
                            rel[k] = moment_rate(k, o->tau[s], o->mrt_rates) * mk / norm;
                        }
                        for (int i = 0; i < 19; ++i) {
                            double back = 0.0;
                            for (int k = 0; k < 19; ++k) back += moment_row(k, CX[i], CY[i], CZ[i]) * rel[k];
                            o->fpost[o->pidx(s, i, n)] = o->fstream[o->pidx(s, i, n)] - back;
                        }
                    }
                }
            }
    o->apply_storage();
}

// Density and velocity of the stored (post-collision) populations (Eq. 6):
// rho_s = sum_i g*_i^s, u = sum_s sum_i g*_i^s c_i / sum_s rho_s.
void orc_fields(void* h, double* rho_a, double* rho_b, double* u) {
    Oracle* o = (Oracle*)h;
    const int64_t N = o->nodes();
    for (int64_t n = 0; n < N; ++n) {
        double r[2] = {0.0, 0.0}, m[3] = {0.0, 0.0, 0.0};
        for (int s = 0; s < 2; ++s)
            for (int i = 0; i < 19; ++i) {
                double f = o->fpost[o->pidx(s, i, n)];
                r[s] += f;
                m[0] += f * CX[i];
                m[1] += f * CY[i];
                m[2] += f * CZ[i];
            }
        rho_a[n] = r[0];
        rho_b[n] = r[1];
        double tot = r[0] + r[1];
        u[3 * n + 0] = m[0] / tot;
        u[3 * n + 1] = m[1] / tot;
        u[3 * n + 2] = m[2] / tot;
    }
}

// Total mass of each component and total momentum of the stored populations.
void orc_checksums(void* h, double* mass, double* mom) {
    Oracle* o = (Oracle*)h;
    const int64_t N = o->nodes();
    mass[0] = mass[1] = 0.0;
    mom[0] = mom[1] = mom[2] = 0.0;
    for (int s = 0; s < 2; ++s)
        for (int i = 0; i < 19; ++i)
            for (int64_t n = 0; n < N; ++n) {
                double f = o->fpost[o->pidx(s, i, n)];
                mass[s] += f;
                mom[0] += f * CX[i];
                mom[1] += f * CY[i];
                mom[2] += f * CZ[i];
            }
}

// Ten FP64 moments of the droplet indicator w = max(phi, 0) with
// phi = (rho_A - rho_B)/(rho_A + rho_B):
// out = {sum w, sum w x, sum w y, sum w z, sum w xx, sum w xy, sum w xz,
//        sum w yy, sum w yz, sum w zz}, coordinates from the box centre.
void orc_moments(void* h, double* out) {
    Oracle* o = (Oracle*)h;
    for (int k = 0; k < 10; ++k) out[k] = 0.0;
    for (int z = 0; z < o->L[2]; ++z)
        for (int y = 0; y < o->L[1]; ++y)
            for (int x = 0; x < o->L[0]; ++x) {
                int64_t n = o->node(x, y, z);
                double r[2] = {0.0, 0.0};
                for (int s = 0; s < 2; ++s)
                    for (int i = 0; i < 19; ++i) r[s] += o->fpost[o->pidx(s, i, n)];
                double phi = (r[0] - r[1]) / (r[0] + r[1]);
                double w = phi > 0.0 ? phi : 0.0;
                double p[3];
                o->position(x, y, z, p);
                out[0] += w;
                out[1] += w * p[0];
                out[2] += w * p[1];
                out[3] += w * p[2];
                out[4] += w * p[0] * p[0];
                out[5] += w * p[0] * p[1];
                out[6] += w * p[0] * p[2];
                out[7] += w * p[1] * p[1];
                out[8] += w * p[1] * p[2];
                out[9] += w * p[2] * p[2];
            }
}

// The lattice tables, exported so tests can check them against the
// moment identities of D3Q19 without retyping them.
void orc_lattice(int* cx, int* cy, int* cz, double* w) {
    for (int i = 0; i < 19; ++i) {
        cx[i] = CX[i]; cy[i] = CY[i]; cz[i] = CZ[i];
        w[i] = weight(i);
    }
}

double orc_equilibrium(int i, double rho, const double* u) { return equilibrium(i, rho, u); }

// Thread count of the node loops; returns the count in effect.
int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

}  // extern "C"
