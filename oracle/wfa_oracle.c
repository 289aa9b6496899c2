/*
 * FP64 CPU oracle for the explicit finite-volume heat / advection-diffusion
 * sweep (arXiv 2209.13768, Sec. 1.1.1, Eq. expl_form, generalised to the
 * conservative face-flux form with harmonic-mean face conductivity and
 * first-order upwind advection).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it. It shares no code, header or constant with the
 * CUDA library.
 *
 * What one step computes (Jacobi / ping-pong: every right-hand side uses
 * step n, as Eq. expl_form does):
 *   acc[C] = 0 for every cell.
 *   For every face between a lower cell C and an upper cell D along axis a
 *   (the face between cell n_a-1 and cell 0 too, when the axis is periodic):
 *     K    = 2 kC kD / (kC + kD)            (0 when kC + kD == 0)
 *     diff = K (T_D - T_C) / h_a^2          (Fourier flux, Eq. diff_eq)
 *     F    = (max(u_a,0) T_C + min(u_a,0) T_D) / h_a   (upwind flux)
 *     acc[C] += diff - F ;  acc[D] += -diff + F
 *   Boundary face of cell C with kind DIRICHLET (value Tb on the face, half
 *   a cell from the centre):
 *     diff = 2 kC (Tb - T_C) / h_a^2, upwind value Tb on inflow, T_C on
 *     outflow; the flux enters the balance like an interior face.
 *   ZEROFLUX faces carry neither diffusive nor advective flux.
 *   DIRICHLET_CELL faces: the outer cell layer is held at the face value
 *     (Eq. expl_form, the cells in "bc"); faces between a held cell and an
 *     interior cell are interior faces.
 *   T'[C] = T[C] + dt acc[C] for every cell that is not held.
 * A cell on several held layers takes the value of the last of them in the
 * face order -x, +x, -y, +y, -z, +z.
 *
 * Layout: dense, x fastest: index = i + nx (j + ny l).
 * Parallel: each pass runs over lines along one axis, so no two threads
 * touch the same accumulator; results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_DIRICHLET = 0, OR_ZEROFLUX = 1, OR_PERIODIC = 2, OR_DIRICHLET_CELL = 3 };
enum { OR_ROUND_NONE = 0, OR_ROUND_F32 = 1, OR_ROUND_BF16 = 2 };

typedef struct {
    int64_t n[3];
    double h[3];
    double u[3];
    double k_uniform;
    const double* k; /* per-cell conductivity (dense), or NULL for k_uniform */
    int kind[6];     /* faces -x,+x,-y,+y,-z,+z */
    double value[6];
    double dt;
} prob_t;

static double kc(const prob_t* p, int64_t c) { return p->k ? p->k[c] : p->k_uniform; }

/* Harmonic mean of two cell conductivities (the face conductivity). */
static double harmonic(double a, double b) {
    double s = a + b;
    return s > 0.0 ? 2.0 * a * b / s : 0.0;
}

static int check(const prob_t* p) {
    for (int a = 0; a < 3; ++a) {
        if (p->n[a] < 1 || !(p->h[a] > 0.0)) return -1;
        int lo = p->kind[2 * a], hi = p->kind[2 * a + 1];
        if (lo < 0 || lo > 3 || hi < 0 || hi > 3) return -1;
        if ((lo == OR_PERIODIC) != (hi == OR_PERIODIC)) return -3;
    }
    return 0;
}

/* Round an fp32 value to bfloat16, round-to-nearest-even on the 16 dropped
 * mantissa bits (the usual bias-and-truncate method); NaN stays NaN. */
static float round_bf16(float f) {
    uint32_t b;
    memcpy(&b, &f, 4);
    if ((b & 0x7f800000u) == 0x7f800000u && (b & 0x007fffffu)) {
        b = (b | 0x00400000u) & 0xffff0000u;
    } else {
        b += 0x7fffu + ((b >> 16) & 1u);
        b &= 0xffff0000u;
    }
    memcpy(&f, &b, 4);
    return f;
}

double wfa_oracle_round(double v, int mode) {
    if (mode == OR_ROUND_F32) return (double)(float)v;
    if (mode == OR_ROUND_BF16) return (double)round_bf16((float)v);
    return v;
}

/* wfa_oracle_round applied to n values in place. */
void wfa_oracle_round_array(double* x, int64_t n, int mode) {
    for (int64_t i = 0; i < n; ++i) x[i] = wfa_oracle_round(x[i], mode);
}

/* Face-flux accumulation along axis a (one pass). */
static void face_pass(const prob_t* p, const double* T, double* acc, int a) {
    const int64_t nx = p->n[0], ny = p->n[1];
    const int64_t st[3] = {1, nx, nx * ny};
    const int64_t na = p->n[a];
    const int b = (a == 0) ? 1 : 0;   /* the two other axes */
    const int c = (a == 2) ? 1 : 2;   /* outer (parallel) axis */
    const double inv_h2 = 1.0 / (p->h[a] * p->h[a]);
    const double inv_h = 1.0 / p->h[a];
    const double up = p->u[a] > 0.0 ? p->u[a] : 0.0;
    const double um = p->u[a] < 0.0 ? p->u[a] : 0.0;
    const int klo = p->kind[2 * a], khi = p->kind[2 * a + 1];
    const double vlo = p->value[2 * a], vhi = p->value[2 * a + 1];
    const int periodic = (klo == OR_PERIODIC);
    const int64_t nb = p->n[b], ncc = p->n[c];

#pragma omp parallel for schedule(static)
    for (int64_t ic = 0; ic < ncc; ++ic) {
        for (int64_t ib = 0; ib < nb; ++ib) {
            const int64_t base = ib * st[b] + ic * st[c];
            /* interior faces, plus the wrap-around face of a periodic axis */
            const int64_t nface = periodic ? (na > 1 ? na : 0) : na - 1;
            for (int64_t i = 0; i < nface; ++i) {
                const int64_t C = base + i * st[a];
                const int64_t D = base + ((i + 1) % na) * st[a];
                const double K = harmonic(kc(p, C), kc(p, D));
                const double diff = K * (T[D] - T[C]) * inv_h2;
                const double F = (up * T[C] + um * T[D]) * inv_h;
                acc[C] += diff - F;
                acc[D] += -diff + F;
            }
            if (!periodic) {
                const int64_t C0 = base;                  /* lower boundary face */
                if (klo == OR_DIRICHLET) {
                    const double diff = 2.0 * kc(p, C0) * (vlo - T[C0]) * inv_h2;
                    const double F = (up * vlo + um * T[C0]) * inv_h;   /* +a flux into C0 */
                    acc[C0] += diff + F;
                }
                const int64_t C1 = base + (na - 1) * st[a];  /* upper boundary face */
                if (khi == OR_DIRICHLET) {
                    const double diff = 2.0 * kc(p, C1) * (vhi - T[C1]) * inv_h2;
                    const double F = (up * T[C1] + um * vhi) * inv_h;   /* +a flux out of C1 */
                    acc[C1] += diff - F;
                }
            }
        }
    }
}

/* held[c] = 1 + index of the face whose layer holds cell c, 0 if updated. */
static unsigned char* held_mask(const prob_t* p) {
    const int64_t nx = p->n[0], ny = p->n[1], nz = p->n[2];
    const int64_t N = nx * ny * nz;
    unsigned char* m = (unsigned char*)calloc((size_t)N, 1);
    if (!m) return NULL;
    for (int f = 0; f < 6; ++f) {
        if (p->kind[f] != OR_DIRICHLET_CELL) continue;
        const int a = f / 2;
        const int64_t want = (f % 2 == 0) ? 0 : p->n[a] - 1;
        for (int64_t l = 0; l < nz; ++l)
            for (int64_t j = 0; j < ny; ++j)
                for (int64_t i = 0; i < nx; ++i) {
                    const int64_t idx[3] = {i, j, l};
                    if (idx[a] == want) m[i + nx * (j + ny * l)] = (unsigned char)(f + 1);
                }
    }
    return m;
}

/*
 * Advance T (dense, nx*ny*nz doubles, in place) by nsteps explicit steps.
 * round_to: 0 none, 1 fp32, 2 bf16 (fp64 -> fp32 -> bf16, both nearest-even),
 * applied after every step (a diagnostic that models storage rounding).
 * Returns 0, -1 on a bad argument, -2 on allocation failure, -3 on a
 * periodic face paired with a non-periodic one.
 */
int wfa_oracle_run(const int64_t n[3], const double h[3], const double u[3], double k_uniform,
                   const double* k, const int kind[6], const double value[6], double dt,
                   double* T, int64_t nsteps, int round_to, int nthreads) {
    prob_t p;
    memcpy(p.n, n, sizeof p.n);
    memcpy(p.h, h, sizeof p.h);
    memcpy(p.u, u, sizeof p.u);
    p.k_uniform = k_uniform;
    p.k = k;
    memcpy(p.kind, kind, sizeof p.kind);
    memcpy(p.value, value, sizeof p.value);
    p.dt = dt;
    int rc = check(&p);
    if (rc) return rc;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    const int64_t N = n[0] * n[1] * n[2];
    double* acc = (double*)malloc((size_t)N * sizeof(double));
    unsigned char* held = held_mask(&p);
    if (!acc || !held) {
        free(acc);
        free(held);
        return -2;
    }
    /* the held layers carry their value at every step, step 0 included */
    for (int64_t c = 0; c < N; ++c)
        if (held[c]) T[c] = wfa_oracle_round(value[held[c] - 1], round_to);
    for (int64_t s = 0; s < nsteps; ++s) {
        memset(acc, 0, (size_t)N * sizeof(double));
        for (int a = 0; a < 3; ++a) face_pass(&p, T, acc, a);
#pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < N; ++c) {
            if (held[c]) continue;
            T[c] = wfa_oracle_round(T[c] + dt * acc[c], round_to);
        }
    }
    free(acc);
    free(held);
    return 0;
}

/*
 * Largest stable (positivity-preserving) time step: the update is
 * T'_C = (1 - dt D_C) T_C + dt * (non-negative weights x neighbour values),
 * so every weight is non-negative iff dt <= 1 / max_C D_C. D_C sums the
 * diffusive face conductances / h^2 (2 kC / h^2 on a Dirichlet face, 0 on a
 * zero-flux face) and |u_a| / h_a for every outflow face that carries flux.
 * Held cells are excluded. Returns +inf when no cell has any coupling.
 * For uniform k = 1, h = 1 and Dirichlet cells on all faces this is 1/6,
 * the "omega < 1/6" limit of Sec. 1.1.1.
 */
double wfa_oracle_dt_max(const int64_t n[3], const double h[3], const double u[3], double k_uniform,
                         const double* k, const int kind[6]) {
    prob_t p;
    memcpy(p.n, n, sizeof p.n);
    memcpy(p.h, h, sizeof p.h);
    memcpy(p.u, u, sizeof p.u);
    p.k_uniform = k_uniform;
    p.k = k;
    memcpy(p.kind, kind, sizeof p.kind);
    for (int f = 0; f < 6; ++f) p.value[f] = 0.0;
    p.dt = 0.0;
    if (check(&p)) return -1.0;
    unsigned char* held = held_mask(&p);
    if (!held) return -2.0;
    const int64_t nx = n[0], ny = n[1], nz = n[2];
    const int64_t st[3] = {1, nx, nx * ny};
    double dmax = 0.0;
    for (int64_t l = 0; l < nz; ++l)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                const int64_t C = i + nx * (j + ny * l);
                if (held[C]) continue;
                const int64_t idx[3] = {i, j, l};
                double D = 0.0;
                for (int a = 0; a < 3; ++a) {
                    const double inv_h2 = 1.0 / (h[a] * h[a]);
                    for (int side = 0; side < 2; ++side) {
                        const int f = 2 * a + side;
                        const int at_edge = side == 0 ? idx[a] == 0 : idx[a] == n[a] - 1;
                        int active = 1;
                        if (kind[f] == OR_PERIODIC && n[a] == 1) {
                            continue; /* a face to itself carries no net flux */
                        } else if (at_edge && kind[f] != OR_PERIODIC) {
                            if (kind[f] == OR_DIRICHLET) D += 2.0 * kc(&p, C) * inv_h2;
                            else active = 0;
                        } else {
                            int64_t ia = idx[a] + (side == 0 ? -1 : 1);
                            ia = (ia + n[a]) % n[a];
                            const int64_t Dn = C + (ia - idx[a]) * st[a];
                            D += harmonic(kc(&p, C), kc(&p, Dn)) * inv_h2;
                        }
                        /* outflow through this face carries T_C away */
                        if (active) {
                            if (side == 1 && u[a] > 0.0) D += u[a] / h[a];
                            if (side == 0 && u[a] < 0.0) D += -u[a] / h[a];
                        }
                    }
                }
                if (D > dmax) dmax = D;
            }
    free(held);
    return dmax > 0.0 ? 1.0 / dmax : INFINITY;
}

/* Total heat E = sum_C T_C hx hy hz (unit heat capacity), plain fp64 sum. */
double wfa_oracle_total_heat(const int64_t n[3], const double h[3], const double* T) {
    const int64_t N = n[0] * n[1] * n[2];
    double s = 0.0;
    for (int64_t c = 0; c < N; ++c) s += T[c];
    return s * h[0] * h[1] * h[2];
}

/*
 * Backward-time, centred-space steps solved by classic conjugate gradients
 * (Sec. 1.1.2, Eq. impl_form, in the face-flux form above; diffusion only:
 * with advection the system is not symmetric and CG does not apply, so u is
 * not an argument).
 *
 * One step finds T^{n+1} with
 *   T^{n+1}_C - dt acc(T^{n+1})_C = T^n_C   for every cell that is not held,
 *   T^{n+1}_C = its face value              for held cells,
 * where acc is the explicit step's accumulation (face_pass), affine in T
 * through the Dirichlet face values. Split T^{n+1} = z + y with z the held
 * values on held cells and 0 elsewhere, y zero on held cells; then on the
 * free cells
 *   A y = b,   A y = y - dt acc0(y),   b = T^n + dt acc(z),
 * acc0 being acc with every Dirichlet face value set to 0 (its linear part).
 * A is symmetric positive definite (unit diagonal plus a weighted graph
 * Laplacian; Eq. impl_form is this system for uniform k and held layers,
 * scaled by psi = 1 / (1 + 6 omega)).
 *
 * Classic CG (Hestenes and Stiefel), two inner products per iteration as in
 * Sec. 1.1.2; every inner product is a plain sequential fp64 sum over the
 * free cells in index order:
 *   x = T^n on free cells;  r = b - A x;  p = r;  rr = r.r;  bb = b.b
 *   while rr > rtol^2 bb and it < max_iter:
 *     q = A p;  alpha = rr / (p.q);  x += alpha p;  r -= alpha q
 *     rr' = r.r;  beta = rr' / rr;  p = r + beta p;  rr = rr';  ++it
 * T^{n+1} = z + x. *iters receives the iterations of all steps together,
 * *rel_res the last step's sqrt(rr / bb) (sqrt(rr) when bb = 0).
 * Returns 0, -1 / -3 like wfa_oracle_run, -2 on allocation failure.
 */
static void apply_A(const prob_t* p0, const unsigned char* held, const double* y, double* out, double* acc) {
    const int64_t N = p0->n[0] * p0->n[1] * p0->n[2];
    memset(acc, 0, (size_t)N * sizeof(double));
    for (int a = 0; a < 3; ++a) face_pass(p0, y, acc, a);
    for (int64_t c = 0; c < N; ++c) out[c] = held[c] ? 0.0 : y[c] - p0->dt * acc[c];
}

static double dot_free(const unsigned char* held, const double* a, const double* b, int64_t N) {
    double s = 0.0;
    for (int64_t c = 0; c < N; ++c)
        if (!held[c]) s += a[c] * b[c];
    return s;
}

int wfa_oracle_implicit(const int64_t n[3], const double h[3], double k_uniform, const double* k,
                        const int kind[6], const double value[6], double dt, double* T, int64_t nsteps,
                        double rtol, int64_t max_iter, int64_t* iters, double* rel_res, int nthreads) {
    prob_t p, p0;
    memcpy(p.n, n, sizeof p.n);
    memcpy(p.h, h, sizeof p.h);
    for (int a = 0; a < 3; ++a) p.u[a] = 0.0;
    p.k_uniform = k_uniform;
    p.k = k;
    memcpy(p.kind, kind, sizeof p.kind);
    memcpy(p.value, value, sizeof p.value);
    p.dt = dt;
    int rc = check(&p);
    if (rc) return rc;
    if (!(dt >= 0.0) || !(rtol >= 0.0) || max_iter < 0) return -1;
    p0 = p;
    for (int f = 0; f < 6; ++f) p0.value[f] = 0.0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    const int64_t N = n[0] * n[1] * n[2];
    unsigned char* held = held_mask(&p);
    double* buf = (double*)malloc((size_t)N * 6 * sizeof(double));
    if (!held || !buf) {
        free(held);
        free(buf);
        return -2;
    }
    double *z = buf, *x = buf + N, *r = buf + 2 * N, *pv = buf + 3 * N, *q = buf + 4 * N, *acc = buf + 5 * N;
    int64_t total = 0;
    double last = 0.0;
    for (int64_t c = 0; c < N; ++c) {
        z[c] = held[c] ? value[held[c] - 1] : 0.0;
        if (held[c]) T[c] = z[c];
    }
    for (int64_t s = 0; s < nsteps; ++s) {
        /* b = T^n + dt acc(z) on the free cells (kept in r for now) */
        memset(acc, 0, (size_t)N * sizeof(double));
        for (int a = 0; a < 3; ++a) face_pass(&p, z, acc, a);
        for (int64_t c = 0; c < N; ++c) {
            r[c] = held[c] ? 0.0 : T[c] + dt * acc[c];
            x[c] = held[c] ? 0.0 : T[c];
        }
        const double bb = dot_free(held, r, r, N);
        apply_A(&p0, held, x, q, acc);
        for (int64_t c = 0; c < N; ++c) {
            r[c] -= q[c];
            pv[c] = r[c];
        }
        double rr = dot_free(held, r, r, N);
        int64_t it = 0;
        while (rr > rtol * rtol * bb && it < max_iter) {
            apply_A(&p0, held, pv, q, acc);
            const double pq = dot_free(held, pv, q, N);
            if (!(pq > 0.0)) break; /* exact solution reached (p = 0) or breakdown */
            const double alpha = rr / pq;
            for (int64_t c = 0; c < N; ++c) {
                x[c] += alpha * pv[c];
                r[c] -= alpha * q[c];
            }
            const double rr_new = dot_free(held, r, r, N);
            const double beta = rr_new / rr;
            for (int64_t c = 0; c < N; ++c) pv[c] = r[c] + beta * pv[c];
            rr = rr_new;
            ++it;
        }
        for (int64_t c = 0; c < N; ++c)
            if (!held[c]) T[c] = x[c];
        total += it;
        last = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
    }
    if (iters) *iters = total;
    if (rel_res) *rel_res = last;
    free(held);
    free(buf);
    return 0;
}

/*
 * The same backward-Euler steps solved by Chronopoulos and Gear's CG: one
 * synchronisation per iteration, both inner products taken together (the
 * reduction-limited Krylov variants Sec. 1.1.2 and Sec. 3.2 point to). In
 * exact arithmetic its iterates are those of classic CG; it carries w = A r
 * and s = A p by recurrence instead of applying A to p:
 *   x = T^n on free cells;  r = b - A x;  w = A r
 *   gamma = r.r;  delta = w.r;  alpha = gamma / delta;  beta = 0
 *   while gamma > rtol^2 bb and it < max_iter:
 *     p = r + beta p;  s = w + beta s
 *     x += alpha p;  r -= alpha s;  w = A r
 *     gamma' = r.r;  delta = w.r
 *     beta = gamma' / gamma;  alpha = gamma' / (delta - beta gamma' / alpha)
 *     gamma = gamma';  ++it
 * Arguments and results as wfa_oracle_implicit.
 */
int wfa_oracle_implicit_cgcg(const int64_t n[3], const double h[3], double k_uniform, const double* k,
                             const int kind[6], const double value[6], double dt, double* T, int64_t nsteps,
                             double rtol, int64_t max_iter, int64_t* iters, double* rel_res, int nthreads) {
    prob_t p, p0;
    memcpy(p.n, n, sizeof p.n);
    memcpy(p.h, h, sizeof p.h);
    for (int a = 0; a < 3; ++a) p.u[a] = 0.0;
    p.k_uniform = k_uniform;
    p.k = k;
    memcpy(p.kind, kind, sizeof p.kind);
    memcpy(p.value, value, sizeof p.value);
    p.dt = dt;
    int rc = check(&p);
    if (rc) return rc;
    if (!(dt >= 0.0) || !(rtol >= 0.0) || max_iter < 0) return -1;
    p0 = p;
    for (int f = 0; f < 6; ++f) p0.value[f] = 0.0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    const int64_t N = n[0] * n[1] * n[2];
    unsigned char* held = held_mask(&p);
    double* buf = (double*)malloc((size_t)N * 7 * sizeof(double));
    if (!held || !buf) {
        free(held);
        free(buf);
        return -2;
    }
    double *z = buf, *x = buf + N, *r = buf + 2 * N, *w = buf + 3 * N, *pv = buf + 4 * N, *sv = buf + 5 * N,
           *acc = buf + 6 * N;
    int64_t total = 0;
    double last = 0.0;
    for (int64_t c = 0; c < N; ++c) {
        z[c] = held[c] ? value[held[c] - 1] : 0.0;
        if (held[c]) T[c] = z[c];
    }
    for (int64_t st = 0; st < nsteps; ++st) {
        memset(acc, 0, (size_t)N * sizeof(double));
        for (int a = 0; a < 3; ++a) face_pass(&p, z, acc, a);
        for (int64_t c = 0; c < N; ++c) {
            r[c] = held[c] ? 0.0 : T[c] + dt * acc[c];   /* b, for now */
            x[c] = held[c] ? 0.0 : T[c];
            pv[c] = sv[c] = 0.0;
        }
        const double bb = dot_free(held, r, r, N);
        apply_A(&p0, held, x, w, acc);
        for (int64_t c = 0; c < N; ++c) r[c] -= w[c];
        apply_A(&p0, held, r, w, acc);
        double gamma = dot_free(held, r, r, N);
        double delta = dot_free(held, w, r, N);
        double alpha = delta > 0.0 ? gamma / delta : 0.0, beta = 0.0;
        int64_t it = 0;
        while (gamma > rtol * rtol * bb && it < max_iter && alpha > 0.0) {
            for (int64_t c = 0; c < N; ++c) {
                pv[c] = r[c] + beta * pv[c];
                sv[c] = w[c] + beta * sv[c];
                x[c] += alpha * pv[c];
                r[c] -= alpha * sv[c];
            }
            apply_A(&p0, held, r, w, acc);
            const double g1 = dot_free(held, r, r, N);
            delta = dot_free(held, w, r, N);
            beta = g1 / gamma;
            const double den = delta - beta * g1 / alpha;
            alpha = den > 0.0 ? g1 / den : 0.0;   /* 0: breakdown or exact solution, the loop ends */
            gamma = g1;
            ++it;
        }
        for (int64_t c = 0; c < N; ++c)
            if (!held[c]) T[c] = x[c];
        total += it;
        last = bb > 0.0 ? sqrt(gamma / bb) : sqrt(gamma);
    }
    if (iters) *iters = total;
    if (rel_res) *rel_res = last;
    free(held);
    free(buf);
    return 0;
}
