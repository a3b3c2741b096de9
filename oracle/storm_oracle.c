/*
 * storm_oracle.c -- FP64 CPU oracle for one STORM sampling-based MPC step.
 *
 * TEST INFRASTRUCTURE ONLY (see storm_oracle.h).  Plain, slow, sequential C in
 * double precision; every loop runs in the order the definition is written.
 * No blocking, fusion or reordering: a reader should be able to hold each
 * routine next to the paper's equation and check it by eye.
 *
 * Parity status of each routine is stated in its comment ("pinned by ...").
 */
#include "storm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Noise: counter-based Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).    */
/* The paper draws Gaussian controls around the mean (Sec. 4, Algorithm 1,    */
/* sample_controls) but fixes no generator; Philox is this project's choice,  */
/* implemented from its published definition.  Pinned by the published        */
/* known-answer vector and, on the GPU, by cuRAND's Philox4_32_10 stream.     */
/* ------------------------------------------------------------------------- */

static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u; /* Weyl key schedule */
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof(c));
}

/* 23 high bits of a word, centred in their cell: never 0, never 1. */
double orc_uniform_from_bits(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Box-Muller transform (Box & Muller 1958). */
void orc_box_muller(double u1, double u2, double* z0, double* z1)
{
    const double r = sqrt(-2.0 * log(u1));
    *z0 = r * cos(2.0 * ORC_PI * u2);
    *z1 = r * sin(2.0 * ORC_PI * u2);
}

/*
 * eps[e], e in [0, count): Philox block e/4 with counter
 * (e/4, step, (instance << 8) | iter, tag) and key (seed lo, seed hi);
 * words (x0, x1) give lanes 0/1 and (x2, x3) lanes 2/3 through Box-Muller.
 */
void orc_noise_philox(uint64_t seed, uint32_t step, uint32_t instance, uint32_t iter,
                      uint32_t tag, long long count, double* eps)
{
    const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (long long e = 0; e < count; ++e) {
        const uint32_t ctr[4] = {(uint32_t)(e / 4), step, (instance << 8) | iter, tag};
        uint32_t x[4];
        orc_philox4x32_10(ctr, key, x);
        const int lane = (int)(e % 4);
        const int pair = lane / 2;
        double z0, z1;
        orc_box_muller(orc_uniform_from_bits(x[2 * pair]),
                       orc_uniform_from_bits(x[2 * pair + 1]), &z0, &z1);
        eps[e] = (lane % 2 == 0) ? z0 : z1;
    }
}

/* ------------------------------------------------------------------------- */
/* Halton low-discrepancy noise (Sec. 4.3, "Sampling Strategy"): point i has  */
/* coordinate phi_{p_k}(i) in the k-th prime base, phi_b(i) = sum_a i_a b^-a. */
/* Reading: unscrambled, point index i = n + 1 (skips i = 0, where the normal */
/* quantile is -inf), dimension k = s*d + j, mapped to N(0,1) by the normal   */
/* quantile, drawn once.  Pinned by exact radical-inverse values.             */
/* ------------------------------------------------------------------------- */

double orc_radical_inverse(uint64_t i, int base)
{
    double f = 1.0 / base, r = 0.0;
    while (i > 0) {
        r += (double)(i % (uint64_t)base) * f;
        i /= (uint64_t)base;
        f /= base;
    }
    return r;
}

int orc_nth_prime(int n) /* n = 0 -> 2 */
{
    int count = -1;
    for (int c = 2;; ++c) {
        int is_prime = 1;
        for (int q = 2; q * q <= c; ++q)
            if (c % q == 0) {
                is_prime = 0;
                break;
            }
        if (is_prime && ++count == n) return c;
    }
}

/* Standard normal quantile: bisection on Phi(x) = erfc(-x/sqrt 2)/2. */
double orc_norm_ppf(double p)
{
    if (!(p > 0.0 && p < 1.0)) return p <= 0.0 ? -INFINITY : INFINITY;
    double lo = -40.0, hi = 40.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (0.5 * erfc(-mid / sqrt(2.0)) < p)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

void orc_noise_halton(int N, int S, int d, double* eps) { orc_noise_halton_ex(N, S, d, 0, 0, eps); }

/* Radical inverse with linearly scrambled digits: digit a of i in base b
 * contributes ((mult * a) mod b) b^-(position).  mult = 1 is the plain
 * radical inverse; for prime b and 0 < mult < b the map is a permutation of
 * the digits that fixes 0 (generalised Halton sequences, Faure and Lemieux). */
double orc_radical_inverse_scrambled(uint64_t i, int base, int mult)
{
    double f = 1.0 / base, r = 0.0;
    while (i > 0) {
        r += (double)(((uint64_t)mult * (i % (uint64_t)base)) % (uint64_t)base) * f;
        i /= (uint64_t)base;
        f /= base;
    }
    return r;
}

/* Multiplier of dimension dim (base b) drawn from the Philox stream of the
 * seed: 1 + (Philox4x32-10 of counter (dim, 0, 0, 3), first word) mod (b - 1). */
int orc_halton_multiplier(uint64_t seed, int dim, int base)
{
    const uint32_t ctr[4] = {(uint32_t)dim, 0u, 0u, 3u};
    const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return base > 2 ? 1 + (int)(out[0] % (uint32_t)(base - 1)) : 1;
}

/* Halton noise (Sec. 4.3): point n + 1 of the sequence in the first S*d primes,
 * mapped to normal by the inverse CDF; scramble selects the linearly scrambled
 * digits (an added option: unscrambled, the first points of the large-prime
 * dimensions are i / p, the same for every such dimension). */
void orc_noise_halton_ex(int N, int S, int d, int scramble, uint64_t seed, double* eps)
{
    for (int n = 0; n < N; ++n)
        for (int s = 0; s < S; ++s)
            for (int j = 0; j < d; ++j) {
                const int dim = s * d + j;
                const int b = orc_nth_prime(dim);
                const int f = scramble ? orc_halton_multiplier(seed, dim, b) : 1;
                const double w = orc_radical_inverse_scrambled((uint64_t)n + 1, b, f);
                eps[((long long)n * S + s) * d + j] = orc_norm_ppf(w);
            }
}

/* ------------------------------------------------------------------------- */
/* Cubic B-spline smoothing (Sec. 4.3): the S sampled knots are the control   */
/* points of a clamped uniform cubic B-spline, evaluated at x_h = h/(H-1).    */
/* Basis by the Cox-de Boor recursion.  Pinned by partition of unity, end     */
/* interpolation and the closed-form uniform cubic blending polynomials.      */
/* ------------------------------------------------------------------------- */

static double knot(int i, int S)
{
    if (i <= 3) return 0.0;
    if (i >= S) return 1.0;
    return (double)(i - 3) / (double)(S - 3);
}

static double cox_de_boor(int i, int p, double x, int S)
{
    if (p == 0) {
        /* right end x = 1 belongs to the last non-empty span [t_{S-1}, t_S) */
        if (x >= 1.0) return (i == S - 1) ? 1.0 : 0.0;
        return (knot(i, S) <= x && x < knot(i + 1, S)) ? 1.0 : 0.0;
    }
    double a = 0.0, b = 0.0;
    const double den_a = knot(i + p, S) - knot(i, S);
    const double den_b = knot(i + p + 1, S) - knot(i + 1, S);
    if (den_a > 0.0) a = (x - knot(i, S)) / den_a * cox_de_boor(i, p - 1, x, S);
    if (den_b > 0.0) b = (knot(i + p + 1, S) - x) / den_b * cox_de_boor(i + 1, p - 1, x, S);
    return a + b;
}

void orc_bspline_basis(int H, int S, double* B)
{
    for (int h = 0; h < H; ++h) {
        const double x = (H > 1) ? (double)h / (double)(H - 1) : 0.0;
        for (int s = 0; s < S; ++s) B[h * S + s] = cox_de_boor(s, 3, x, S);
    }
}

/* u_{n,h} = mu_h + sigma o (B eps_n)_h ; null particles get u = 0 (Sec. 4.3). */
/* Samples per particle and joint drawn for one iteration: the knots of the
 * B-spline, or one per horizon step (no smoothing, comb and mixed filters). */
static int noise_samples(const orc_params* P)
{
    if (P->filter == ORC_FILTER_DEFAULT && P->n_knots > 0) return P->n_knots;
    return P->H;
}

/* Comb filter along the horizon (Sec. 4.3): out_h = c1 eps_h + c2 out_{h-1} +
 * c3 out_{h-2}.  Readings: the printed third term repeats index h-1 and is read
 * as h-2; the recursion runs over the already filtered values (the in-place
 * update the formula describes); values before h = 0 are zero.  eps, out: H x d. */
void orc_comb_filter(int H, int d, const double* c, const double* eps, double* out)
{
    for (int j = 0; j < d; ++j)
        for (int h = 0; h < H; ++h) {
            const double y1 = h >= 1 ? out[(h - 1) * d + j] : 0.0;
            const double y2 = h >= 2 ? out[(h - 2) * d + j] : 0.0;
            out[h * d + j] = c[0] * eps[h * d + j] + c[1] * y1 + c[2] * y2;
        }
}

/* sample_controls (Algorithm 1, Sec. 4.3): u = mu + sigma o smooth(eps), with
 * the filter of P->filter; particles 0..n_null-1 are the zero-acceleration
 * ("null") particles.  eps: N x S x d with S = noise_samples(P). */
void orc_smooth_controls(const orc_params* P, int d, const double* mu, const double* sigma,
                         const double* eps, double* u)
{
    const int N = P->N, H = P->H, S = noise_samples(P), K = P->n_knots;
    double* B = NULL;
    if (K > 0 && P->filter != ORC_FILTER_COMB) {
        B = (double*)malloc(sizeof(double) * H * K);
        orc_bspline_basis(H, K, B);
    }
    const int n_bs = P->filter == ORC_FILTER_MIXED ? (int)floor(P->mix_bspline * (N - P->n_null) + 0.5) : 0;
    double* filt = (double*)malloc(sizeof(double) * H * d);
    for (int n = 0; n < N; ++n) {
        const double* en = eps + (long long)n * S * d;
        int use_bs = 0, use_comb = 0;
        if (P->filter == ORC_FILTER_DEFAULT) use_bs = K > 0;
        else if (P->filter == ORC_FILTER_COMB) use_comb = 1;
        else {
            use_bs = n >= P->n_null && n < P->n_null + n_bs;
            use_comb = !use_bs;
        }
        if (use_comb) orc_comb_filter(H, d, P->comb, en, filt);
        for (int h = 0; h < H; ++h)
            for (int j = 0; j < d; ++j) {
                double e;
                if (use_bs) {
                    e = 0.0;
                    for (int s = 0; s < K; ++s) e += B[h * K + s] * en[s * d + j];
                } else if (use_comb) {
                    e = filt[h * d + j];
                } else {
                    e = en[h * d + j];
                }
                const long long idx = ((long long)n * H + h) * d + j;
                u[idx] = (n < P->n_null) ? 0.0 : mu[h * d + j] + sigma[j] * e;
            }
    }
    free(filt);
    free(B);
}

/* ------------------------------------------------------------------------- */
/* Tensorised integration, Eq. 7: theta_ddot = u,                              */
/* theta_dot = theta_dot_init + S_l(1) diag(dt) theta_ddot,                    */
/* theta = theta_init + S_l(1) diag(dt) theta_dot, with S_l(1) the inclusive   */
/* lower-triangular matrix of ones (written out as its product).  Pinned by    */
/* the constant-acceleration closed form.                                      */
/* ------------------------------------------------------------------------- */
void orc_integrate(int H, int d, const double* dt, const double* state, const double* u,
                   double* theta, double* theta_dot)
{
    for (int j = 0; j < d; ++j) {
        for (int h = 0; h < H; ++h) {
            double v = state[d + j];
            for (int k = 0; k < H; ++k) {
                const double S_l = (k <= h) ? 1.0 : 0.0;
                v += S_l * dt[k] * u[k * d + j];
            }
            theta_dot[h * d + j] = v;
        }
        for (int h = 0; h < H; ++h) {
            double q = state[j];
            for (int k = 0; k < H; ++k) {
                const double S_l = (k <= h) ? 1.0 : 0.0;
                q += S_l * dt[k] * theta_dot[k * d + j];
            }
            theta[h * d + j] = q;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Forward kinematics, Eq. 8: X = FK(theta).  Modified DH (Craig):            */
/* T_i = T_{i-1} RotX(alpha_{i-1}) TransX(a_{i-1}) RotZ(theta_i+off_i)        */
/* TransZ(d_i), T_0 = I; the end-effector frame is T_d.  frames holds         */
/* (d+1) row-major 4x4 matrices.  Pinned by the zero-configuration closed     */
/* form, single-joint Rodrigues rotation and orthonormality.                  */
/* ------------------------------------------------------------------------- */

static void mat4_mul(const double* A, const double* B, double* C)
{
    double T[16];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += A[r * 4 + k] * B[k * 4 + c];
            T[r * 4 + c] = s;
        }
    memcpy(C, T, sizeof(T));
}

static void mat4_identity(double* A)
{
    memset(A, 0, 16 * sizeof(double));
    A[0] = A[5] = A[10] = A[15] = 1.0;
}

static void rot_x(double a, double* A)
{
    mat4_identity(A);
    A[5] = cos(a);
    A[6] = -sin(a);
    A[9] = sin(a);
    A[10] = cos(a);
}

static void rot_z(double a, double* A)
{
    mat4_identity(A);
    A[0] = cos(a);
    A[1] = -sin(a);
    A[4] = sin(a);
    A[5] = cos(a);
}

static void trans(double x, double y, double z, double* A)
{
    mat4_identity(A);
    A[3] = x;
    A[7] = y;
    A[11] = z;
}

void orc_fk(const orc_robot* R, const double* theta, double* frames)
{
    const int d = R->dof;
    mat4_identity(frames);
    for (int i = 1; i <= d; ++i) {
        const double* row = R->dh + (i - 1) * 4; /* a_{i-1}, alpha_{i-1}, d_i, offset_i */
        double Ra[16], Ta[16], Rt[16], Td[16], A[16];
        rot_x(row[1], Ra);
        trans(row[0], 0.0, 0.0, Ta);
        rot_z(theta[i - 1] + row[3], Rt);
        trans(0.0, 0.0, row[2], Td);
        mat4_mul(Ra, Ta, A);
        mat4_mul(A, Rt, A);
        mat4_mul(A, Td, A);
        mat4_mul(frames + (i - 1) * 16, A, frames + i * 16);
    }
}

/* Geometric Jacobian, Eq. 8: column i = [z_i x (p_ee - o_i); z_i] in the world
 * frame, z_i / o_i the axis and origin of joint frame i.  J is 6 x d. Pinned by
 * central finite differences of orc_fk. */
void orc_jacobian(const orc_robot* R, const double* frames, double* J)
{
    const int d = R->dof;
    const double* Te = frames + d * 16;
    const double p[3] = {Te[3], Te[7], Te[11]};
    for (int i = 1; i <= d; ++i) {
        const double* T = frames + i * 16;
        const double z[3] = {T[2], T[6], T[10]};
        const double r[3] = {p[0] - T[3], p[1] - T[7], p[2] - T[11]};
        const int c = i - 1;
        J[0 * d + c] = z[1] * r[2] - z[2] * r[1];
        J[1 * d + c] = z[2] * r[0] - z[0] * r[2];
        J[2 * d + c] = z[0] * r[1] - z[1] * r[0];
        J[3 * d + c] = z[0];
        J[4 * d + c] = z[1];
        J[5 * d + c] = z[2];
    }
}

/* End-effector velocity and acceleration, Eq. 8: X_dot = J theta_dot and
 * X_ddot = J_dot theta_dot + J theta_ddot, both as [linear; angular] about the
 * end-effector point.  J_dot by columns: with z_i, o_i the axis and origin of
 * joint i, w_{i-1} = sum_{k<i} theta_dot_k z_k the angular velocity of the link
 * before it, z_i_dot = w_{i-1} x z_i, o_i_dot = sum_{k<i} theta_dot_k z_k x
 * (o_i - o_k) and p_dot the linear part of X_dot, column i of J_dot is
 * [z_i_dot x (p - o_i) + z_i x (p_dot - o_i_dot); z_i_dot]. */
void orc_ee_twist(const orc_robot* R, const double* frames, const double* theta_dot,
                  const double* theta_ddot, double* xd, double* xdd)
{
    const int d = R->dof;
    double J[6 * 8];
    orc_jacobian(R, frames, J);
    for (int r = 0; r < 6; ++r) {
        xd[r] = 0.0;
        for (int c = 0; c < d; ++c) xd[r] += J[r * d + c] * theta_dot[c];
    }
    const double* Te = frames + d * 16;
    const double p[3] = {Te[3], Te[7], Te[11]};
    double w[3] = {0.0, 0.0, 0.0};
    for (int r = 0; r < 6; ++r) xdd[r] = 0.0;
    for (int c = 0; c < d; ++c) {
        const double* T = frames + (c + 1) * 16;
        const double z[3] = {T[2], T[6], T[10]}, o[3] = {T[3], T[7], T[11]};
        const double zd[3] = {w[1] * z[2] - w[2] * z[1], w[2] * z[0] - w[0] * z[2], w[0] * z[1] - w[1] * z[0]};
        double od[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < c; ++k) {
            const double* Tk = frames + (k + 1) * 16;
            const double zk[3] = {Tk[2], Tk[6], Tk[10]};
            const double r[3] = {o[0] - Tk[3], o[1] - Tk[7], o[2] - Tk[11]};
            od[0] += theta_dot[k] * (zk[1] * r[2] - zk[2] * r[1]);
            od[1] += theta_dot[k] * (zk[2] * r[0] - zk[0] * r[2]);
            od[2] += theta_dot[k] * (zk[0] * r[1] - zk[1] * r[0]);
        }
        const double r[3] = {p[0] - o[0], p[1] - o[1], p[2] - o[2]};
        const double q[3] = {xd[0] - od[0], xd[1] - od[1], xd[2] - od[2]};
        const double jd[3] = {zd[1] * r[2] - zd[2] * r[1] + z[1] * q[2] - z[2] * q[1],
                              zd[2] * r[0] - zd[0] * r[2] + z[2] * q[0] - z[0] * q[2],
                              zd[0] * r[1] - zd[1] * r[0] + z[0] * q[1] - z[1] * q[0]};
        for (int a = 0; a < 3; ++a) {
            xdd[a] += jd[a] * theta_dot[c] + J[a * d + c] * theta_ddot[c];
            xdd[3 + a] += zd[a] * theta_dot[c] + z[a] * theta_ddot[c];
        }
        for (int a = 0; a < 3; ++a) w[a] += theta_dot[c] * z[a];
    }
}

/* Ball on the tray (appendix, ball balancing): the ball's state in the
 * end-effector frame at the current robot state, x0 = T_ee^-1 x_w and
 * v0 = R_ee^T v_w with its normal component zeroed, then per horizon step the
 * in-plane gravity a_h = [g_ee,x, g_ee,y, 0], g_ee = R_ee,h^T g_w, integrated by
 * the same tensorised model as the joints (Eq. 7): v_h = v0 + sum_{k<=h} dt_k a_k,
 * x_h = x0 + sum_{k<=h} dt_k v_k.  theta: H x d; outputs H x 3.  -1 without a ball. */
int orc_ball_states(const orc_robot* R, const orc_params* P, const double* state,
                    const double* theta, double* x_ball, double* v_ball)
{
    if (!P->ball) return -1;
    const int d = R->dof, H = P->H;
    double* frames = (double*)malloc(sizeof(double) * 16 * (d + 1));
    double* a = (double*)malloc(sizeof(double) * 3 * H);
    orc_fk(R, state, frames);
    const double* T0 = frames + d * 16;
    double x0[3], v0[3];
    for (int i = 0; i < 3; ++i) {
        x0[i] = 0.0;
        v0[i] = 0.0;
        for (int k = 0; k < 3; ++k) {
            x0[i] += T0[k * 4 + i] * (P->ball[k] - T0[k * 4 + 3]);
            v0[i] += T0[k * 4 + i] * P->ball[3 + k];
        }
    }
    v0[2] = 0.0;
    for (int h = 0; h < H; ++h) {
        orc_fk(R, theta + (size_t)h * d, frames);
        const double* T = frames + d * 16;
        for (int i = 0; i < 2; ++i) {
            a[h * 3 + i] = 0.0;
            for (int k = 0; k < 3; ++k) a[h * 3 + i] += T[k * 4 + i] * P->gravity[k];
        }
        a[h * 3 + 2] = 0.0;
    }
    for (int h = 0; h < H; ++h)
        for (int i = 0; i < 3; ++i) {
            double v = v0[i];
            for (int k = 0; k <= h; ++k) v += P->dt[k] * a[k * 3 + i];
            v_ball[h * 3 + i] = v;
        }
    for (int h = 0; h < H; ++h)
        for (int i = 0; i < 3; ++i) {
            double x = x0[i];
            for (int k = 0; k <= h; ++k) x += P->dt[k] * v_ball[k * 3 + i];
            x_ball[h * 3 + i] = x;
        }
    free(a);
    free(frames);
    return 0;
}

/* Determinant by LU with partial pivoting. */
double orc_det(int n, const double* A)
{
    double M[64];
    memcpy(M, A, sizeof(double) * n * n);
    double det = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(M[r * n + c]) > fabs(M[piv * n + c])) piv = r;
        if (M[piv * n + c] == 0.0) return 0.0;
        if (piv != c) {
            for (int k = 0; k < n; ++k) {
                const double t = M[c * n + k];
                M[c * n + k] = M[piv * n + k];
                M[piv * n + k] = t;
            }
            det = -det;
        }
        det *= M[c * n + c];
        for (int r = c + 1; r < n; ++r) {
            const double f = M[r * n + c] / M[c * n + c];
            for (int k = c; k < n; ++k) M[r * n + k] -= f * M[c * n + k];
        }
    }
    return det;
}

/* Manipulability score (Sec. 4.2, Eq. 12; Yoshikawa): sqrt(det(J J^T)).
 * Reading: the garbled "sqrt(J J^T)" is the square root of the determinant. */
double orc_manipulability(const double* J, int d)
{
    double JJt[36];
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s += J[r * d + k] * J[c * d + k];
            JJt[r * 6 + c] = s;
        }
    const double det = orc_det(6, JJt);
    return sqrt(det > 0.0 ? det : 0.0);
}

/* Rotation matrix -> unit quaternion (w, x, y, z), Shepperd's method. */
void orc_quat_from_rot(const double* Rm, double* q)
{
    const double m00 = Rm[0], m01 = Rm[1], m02 = Rm[2];
    const double m10 = Rm[3], m11 = Rm[4], m12 = Rm[5];
    const double m20 = Rm[6], m21 = Rm[7], m22 = Rm[8];
    const double tr = m00 + m11 + m22;
    if (tr >= m00 && tr >= m11 && tr >= m22) {
        const double s = 2.0 * sqrt(1.0 + tr);
        q[0] = 0.25 * s;
        q[1] = (m21 - m12) / s;
        q[2] = (m02 - m20) / s;
        q[3] = (m10 - m01) / s;
    } else if (m00 >= m11 && m00 >= m22) {
        const double s = 2.0 * sqrt(1.0 + m00 - m11 - m22);
        q[0] = (m21 - m12) / s;
        q[1] = 0.25 * s;
        q[2] = (m01 + m10) / s;
        q[3] = (m02 + m20) / s;
    } else if (m11 >= m22) {
        const double s = 2.0 * sqrt(1.0 + m11 - m00 - m22);
        q[0] = (m02 - m20) / s;
        q[1] = (m01 + m10) / s;
        q[2] = 0.25 * s;
        q[3] = (m12 + m21) / s;
    } else {
        const double s = 2.0 * sqrt(1.0 + m22 - m00 - m11);
        q[0] = (m10 - m01) / s;
        q[1] = (m02 + m20) / s;
        q[2] = (m12 + m21) / s;
        q[3] = 0.25 * s;
    }
}

/* Unit quaternion (w, x, y, z), normalised first -> rotation matrix. */
void orc_rot_from_quat(const double* q_in, double* Rm)
{
    const double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] +
                          q_in[3] * q_in[3]);
    const double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    Rm[0] = 1 - 2 * (y * y + z * z);
    Rm[1] = 2 * (x * y - w * z);
    Rm[2] = 2 * (x * z + w * y);
    Rm[3] = 2 * (x * y + w * z);
    Rm[4] = 1 - 2 * (x * x + z * z);
    Rm[5] = 2 * (y * z - w * x);
    Rm[6] = 2 * (x * z - w * y);
    Rm[7] = 2 * (y * z + w * x);
    Rm[8] = 1 - 2 * (x * x + y * y);
}

/* ------------------------------------------------------------------------- */
/* Collision (Sec. 4.2, Eqs. 13-14).  The paper's learned self-collision      */
/* network and point-cloud classifier are replaced by exact link-sphere       */
/* geometry.  Reading: signed distance positive when apart; the cost is the   */
/* penetration depth max(0, -min sd).  Self pairs are given as a list.        */
/* Pinned by brute force over a dense box-surface grid and on-axis cases.     */
/* ------------------------------------------------------------------------- */

static void sphere_center(const orc_robot* R, const double* frames, int s, double* c)
{
    const double* T = frames + R->sphere_link[s] * 16;
    const double* p = R->sphere + s * 4;
    for (int r = 0; r < 3; ++r)
        c[r] = T[r * 4 + 0] * p[0] + T[r * 4 + 1] * p[1] + T[r * 4 + 2] * p[2] + T[r * 4 + 3];
}

/* Exact signed distance from point p to an axis-aligned box (negative inside). */
double orc_box_sdf(const double* p, const double* box)
{
    double q[3], out = 0.0, inside = -INFINITY;
    for (int k = 0; k < 3; ++k) {
        q[k] = fabs(p[k] - box[k]) - box[3 + k];
        const double pos = q[k] > 0.0 ? q[k] : 0.0;
        out += pos * pos;
        if (q[k] > inside) inside = q[k];
    }
    return sqrt(out) + (inside < 0.0 ? inside : 0.0);
}

double orc_self_min_sd(const orc_robot* R, const double* frames)
{
    double best = INFINITY;
    for (int k = 0; k < R->n_pairs; ++k) {
        const int a = R->pairs[2 * k], b = R->pairs[2 * k + 1];
        double ca[3], cb[3];
        sphere_center(R, frames, a, ca);
        sphere_center(R, frames, b, cb);
        const double dist = sqrt((ca[0] - cb[0]) * (ca[0] - cb[0]) +
                                 (ca[1] - cb[1]) * (ca[1] - cb[1]) +
                                 (ca[2] - cb[2]) * (ca[2] - cb[2]));
        const double sd = dist - R->sphere[a * 4 + 3] - R->sphere[b * 4 + 3];
        if (sd < best) best = sd;
    }
    return best;
}

double orc_world_min_sd(const orc_robot* R, const orc_world* W, const double* frames)
{
    double best = INFINITY;
    for (int s = 0; s < R->n_spheres; ++s) {
        double c[3];
        sphere_center(R, frames, s, c);
        const double r = R->sphere[s * 4 + 3];
        for (int b = 0; b < W->n_boxes; ++b) {
            const double sd = orc_box_sdf(c, W->boxes + b * 6) - r;
            if (sd < best) best = sd;
        }
        for (int o = 0; o < W->n_spheres; ++o) {
            const double* S = W->spheres + o * 4;
            const double dist = sqrt((c[0] - S[0]) * (c[0] - S[0]) + (c[1] - S[1]) * (c[1] - S[1]) +
                                     (c[2] - S[2]) * (c[2] - S[2]));
            const double sd = dist - r - S[3];
            if (sd < best) best = sd;
        }
    }
    return best;
}

/* ------------------------------------------------------------------------- */
/* Running cost, Eq. 15, with the terms of Eqs. 9-14:                         */
/*  pos   (Eq. 9)  || alpha_2 o R_g^T (d_ee - d_g) ||_2                        */
/*  rot   (Eq. 9)  QUAT: 1 - |q_ee . q_g|; FROBENIUS: ||(I - R_g^T R_ee) diag(alpha_1)||_F */
/*  stop  (Eq. 10) || max(0, |theta_dot| - theta_dot_max,h) ||_2 with         */
/*                 theta_dot_max = S_u(1) qdd_max dt (inclusive upper ones)    */
/*  joint (Eq. 11) || max(0, th_min' - theta) + max(0, theta - th_max') ||_2  */
/*  manip (Eq. 12) (1 - m) if m < k_m else 0, m = sqrt(det J J^T)             */
/*  self/world (Eqs. 13-14) penetration depths of the link spheres            */
/*  smooth        ||u_h - u_{h-1}||^2, u_{-1} = theta_ddot_init (not in the   */
/*                paper; a configurable extra term, weight 0 disables it)     */
/* terms[ORC_NTERMS] receives the unweighted terms in that order.             */
/* ------------------------------------------------------------------------- */
void orc_running_cost(const orc_robot* R, const orc_world* W, const orc_params* P,
                      const double* goal, int h, const double* theta_h,
                      const double* theta_dot_h, const double* u_h, const double* u_prev,
                      double* terms, double* total)
{
    const int d = R->dof, H = P->H;
    double* frames = (double*)malloc(sizeof(double) * 16 * (d + 1));
    double J[6 * 8];
    orc_fk(R, theta_h, frames);
    orc_jacobian(R, frames, J);
    const double* Te = frames + d * 16;
    const double Ree[9] = {Te[0], Te[1], Te[2], Te[4], Te[5], Te[6], Te[8], Te[9], Te[10]};
    double Rg[9];
    orc_rot_from_quat(goal + 3, Rg);

    /* position: R_g^T (d_ee - d_g), weighted per goal-frame axis */
    const double dp[3] = {Te[3] - goal[0], Te[7] - goal[1], Te[11] - goal[2]};
    double c_pos = 0.0;
    for (int i = 0; i < 3; ++i) {
        const double e = Rg[0 * 3 + i] * dp[0] + Rg[1 * 3 + i] * dp[1] + Rg[2 * 3 + i] * dp[2];
        c_pos += (P->pos_axis_w[i] * e) * (P->pos_axis_w[i] * e);
    }
    c_pos = sqrt(c_pos);

    double c_rot = 0.0;
    if (P->rot_mode == ORC_ROT_QUAT) {
        double qe[4], qg[4];
        orc_quat_from_rot(Ree, qe);
        const double ng = sqrt(goal[3] * goal[3] + goal[4] * goal[4] + goal[5] * goal[5] +
                               goal[6] * goal[6]);
        for (int i = 0; i < 4; ++i) qg[i] = goal[3 + i] / ng;
        c_rot = 1.0 - fabs(qe[0] * qg[0] + qe[1] * qg[1] + qe[2] * qg[2] + qe[3] * qg[3]);
    } else {
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double RtR = 0.0;
                for (int k = 0; k < 3; ++k) RtR += Rg[k * 3 + r] * Ree[k * 3 + c];
                const double E = ((r == c) ? 1.0 : 0.0) - RtR;
                c_rot += (E * P->rot_axis_w[c]) * (E * P->rot_axis_w[c]);
            }
        c_rot = sqrt(c_rot);
    }

    double vmax = 0.0; /* (S_u(1) qdd_max dt)_h */
    for (int k = 0; k < H; ++k) vmax += (k >= h ? 1.0 : 0.0) * P->qdd_max * P->dt[k];
    double c_stop = 0.0, c_joint = 0.0, c_smooth = 0.0;
    for (int j = 0; j < d; ++j) {
        const double vs = fabs(theta_dot_h[j]) - vmax;
        if (vs > 0.0) c_stop += vs * vs;
        const double range = R->q_max[j] - R->q_min[j];
        const double lo = R->q_min[j] + P->k_jl * range;
        const double hi = R->q_max[j] - P->k_jl * range;
        const double vj = (theta_h[j] < lo ? lo - theta_h[j] : 0.0) +
                          (theta_h[j] > hi ? theta_h[j] - hi : 0.0);
        c_joint += vj * vj;
        const double du = u_h[j] - u_prev[j];
        c_smooth += du * du;
    }
    c_stop = sqrt(c_stop);
    c_joint = sqrt(c_joint);

    const double m = orc_manipulability(J, d);
    const double c_manip = (m < P->k_m) ? 1.0 - m : 0.0;

    const double sd_self = orc_self_min_sd(R, frames);
    const double sd_world = orc_world_min_sd(R, W, frames);
    double c_self = sd_self < 0.0 ? -sd_self : 0.0;
    if (P->mlp_mode != 0) {
        /* the learned network of Sec. 4.2 on this configuration, with the BF16
         * rounding of a tensor-core forward pass */
        const orc_mlp_arch A = {P->mlp_enc, P->mlp_h1, P->mlp_h2, P->mlp_h3};
        double y = 0.0;
        orc_mlp_arch_forward(&A, P->mlp_params, theta_h, 1, d, 1, &y);
        if (P->mlp_mode == 2)
            c_self = y > 0.0 ? y : 0.0;  /* Eq. 13: the network's depth is the cost */
        else if (y >= P->mlp_margin)
            c_self = 0.0;  /* predicted clear by the margin: the exact check is skipped */
    }
    const double c_world = sd_world < 0.0 ? -sd_world : 0.0;

    /* task-space speed and acceleration limits on Eq. 8's X_dot, X_ddot (theta_ddot = u) */
    double xd[6], xdd[6];
    orc_ee_twist(R, frames, theta_dot_h, u_h, xd, xdd);
    const double speed = sqrt(xd[0] * xd[0] + xd[1] * xd[1] + xd[2] * xd[2]);
    const double accel = sqrt(xdd[0] * xdd[0] + xdd[1] * xdd[1] + xdd[2] * xdd[2]);
    const double c_eev = speed > P->ee_vel_max ? speed - P->ee_vel_max : 0.0;
    const double c_eea = accel > P->ee_acc_max ? accel - P->ee_acc_max : 0.0;

    terms[0] = c_pos;
    terms[1] = c_rot;
    terms[2] = c_stop;
    terms[3] = c_joint;
    terms[4] = c_manip;
    terms[5] = c_self;
    terms[6] = c_world;
    terms[7] = c_smooth;
    terms[8] = c_eev;
    terms[9] = c_eea;
    terms[10] = 0.0;  /* the ball term needs the whole rollout: orc_rollout */
    *total = P->w_pos * c_pos + P->w_rot * c_rot + P->w_stop * c_stop + P->w_joint * c_joint +
             P->w_manip * c_manip + P->w_coll * (c_self + c_world) + P->w_smooth * c_smooth +
             P->w_ee_vel * c_eev + P->w_ee_acc * c_eea;
    free(frames);
}

/* ------------------------------------------------------------------------- */
/* generate_rollouts (Algorithm 1) for one optimisation iteration: controls,  */
/* integration (Eq. 7), per-step costs (Eq. 15) and the discounted total      */
/* C_n = sum_h gamma^h c_{n,h} (Eq. 2, terminal cost read as the running cost */
/* at h = H-1).  Any output pointer may be NULL.                              */
/*   ee: N x H x 12 (row-major 3x4 [R | p]); terms: N x H x ORC_NTERMS         */
/* ------------------------------------------------------------------------- */
/* Host threads of orc_rollout's particle loop (1 = sequential).  Particles are
 * independent and each writes only its own outputs, and no reduction crosses
 * particles, so every thread count gives bitwise the sequential results. */
static int g_orc_threads = 1;

void orc_set_threads(int n) { g_orc_threads = n < 1 ? 1 : n; }
int orc_get_threads(void) { return g_orc_threads; }

int orc_rollout(const orc_robot* R, const orc_world* W, const orc_params* P,
                const double* state, const double* goal, const double* mu,
                const double* sigma, const double* eps, double* u_out, double* theta_out,
                double* theta_dot_out, double* ee_out, double* terms_out, double* cost_out,
                double* Ctot)
{
    const int N = P->N, H = P->H, d = R->dof;
    if (N <= 0 || H <= 0 || d <= 0 || d > 8) return -1;
    double* u = (double*)malloc(sizeof(double) * (size_t)N * H * d);
    orc_smooth_controls(P, d, mu, sigma, eps, u);
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_orc_threads) if (g_orc_threads > 1)
    for (int n = 0; n < N; ++n) {
        double* th = (double*)malloc(sizeof(double) * (size_t)H * d);
        double* thd = (double*)malloc(sizeof(double) * (size_t)H * d);
        double* frames = (double*)malloc(sizeof(double) * 16 * (d + 1));
        double* xb = (double*)malloc(sizeof(double) * 3 * H);
        double* vb = (double*)malloc(sizeof(double) * 3 * H);
        const double* un = u + (size_t)n * H * d;
        orc_integrate(H, d, P->dt, state, un, th, thd);
        const int with_ball = P->w_ball != 0.0 && P->ball;
        if (with_ball) orc_ball_states(R, P, state, th, xb, vb);
        double C = 0.0;
        for (int h = 0; h < H; ++h) {
            double terms[ORC_NTERMS], c;
            const double* uprev = (h == 0) ? state + 2 * d : un + (h - 1) * d;
            orc_running_cost(R, W, P, goal, h, th + h * d, thd + h * d, un + h * d, uprev, terms,
                             &c);
            if (with_ball) {  /* distance of the ball from the tray centre, in the tray plane */
                const double ex = xb[h * 3] - P->tray_center[0], ey = xb[h * 3 + 1] - P->tray_center[1];
                terms[10] = sqrt(ex * ex + ey * ey);
                c += P->w_ball * terms[10];
            }
            C += pow(P->gamma, (double)h) * c;
            const size_t nh = (size_t)n * H + h;
            if (terms_out) memcpy(terms_out + nh * ORC_NTERMS, terms, sizeof(terms));
            if (cost_out) cost_out[nh] = c;
            if (ee_out) {
                orc_fk(R, th + h * d, frames);
                const double* Te = frames + d * 16;
                for (int k = 0; k < 12; ++k) ee_out[nh * 12 + k] = Te[k];
            }
        }
        if (theta_out) memcpy(theta_out + (size_t)n * H * d, th, sizeof(double) * H * d);
        if (theta_dot_out) memcpy(theta_dot_out + (size_t)n * H * d, thd, sizeof(double) * H * d);
        if (Ctot) Ctot[n] = C;
        free(th);
        free(thd);
        free(frames);
        free(xb);
        free(vb);
    }
    if (u_out) memcpy(u_out, u, sizeof(double) * (size_t)N * H * d);
    free(u);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* update_distribution, Eqs. 4-6.  w_i = exp(-C_i / beta), evaluated as       */
/* exp(-(C_i - min C)/beta) (the common factor cancels in the normalised      */
/* weights).  mu <- (1-a_mu) mu + a_mu sum w u / sum w;                        */
/* sigma_j^2 <- (1-a_s) sigma_j^2 + a_s (1/H) sum_h sum_i w (u - mu_new)^2 /   */
/* sum w (diagonal, shared over the horizon: Sec. 4.3 covariance              */
/* parameterisation); sigma_j >= sigma_min.  beta = 0 selects the argmin      */
/* (lowest index on ties); non-finite costs get weight 0.  Returns 1 and      */
/* leaves mu, sigma unchanged if no cost is finite.  Pinned by the MPPI       */
/* special cases (one particle, zero temperature, equal costs, unit sum).     */
/* ------------------------------------------------------------------------- */
int orc_update(const orc_params* P, int d, const double* Ctot, const double* u, double* mu,
               double* sigma, double* weights)
{
    const int N = P->N, H = P->H;
    double m = INFINITY;
    int arg = -1;
    for (int n = 0; n < N; ++n)
        if (isfinite(Ctot[n]) && Ctot[n] < m) {
            m = Ctot[n];
            arg = n;
        }
    if (arg < 0) return 1;
    double* w = (double*)malloc(sizeof(double) * N);
    double s = 0.0;
    for (int n = 0; n < N; ++n) {
        if (!isfinite(Ctot[n]))
            w[n] = 0.0;
        else if (P->beta > 0.0)
            w[n] = exp(-(Ctot[n] - m) / P->beta);
        else
            w[n] = (n == arg) ? 1.0 : 0.0;
        s += w[n];
    }
    for (int n = 0; n < N; ++n) w[n] /= s;
    for (int h = 0; h < H; ++h)
        for (int j = 0; j < d; ++j) {
            double acc = 0.0;
            for (int n = 0; n < N; ++n) acc += w[n] * u[((size_t)n * H + h) * d + j];
            mu[h * d + j] = (1.0 - P->alpha_mu) * mu[h * d + j] + P->alpha_mu * acc;
        }
    for (int j = 0; j < d; ++j) {
        double acc = 0.0;
        for (int h = 0; h < H; ++h)
            for (int n = 0; n < N; ++n) {
                const double e = u[((size_t)n * H + h) * d + j] - mu[h * d + j];
                acc += w[n] * e * e;
            }
        double var = (1.0 - P->alpha_sigma) * sigma[j] * sigma[j] + P->alpha_sigma * acc / H;
        if (var < P->sigma_min * P->sigma_min) var = P->sigma_min * P->sigma_min;
        sigma[j] = sqrt(var);
    }
    if (weights) memcpy(weights, w, sizeof(double) * N);
    free(w);
    return 0;
}

/* shift (Algorithm 1, Sec. 4): mu_h <- mu_{h+1}; the appended default is zero
 * acceleration.  The per-joint sigma is left as it is. */
void orc_shift(int H, int d, double* mu)
{
    for (int h = 0; h + 1 < H; ++h)
        for (int j = 0; j < d; ++j) mu[h * d + j] = mu[(h + 1) * d + j];
    for (int j = 0; j < d; ++j) mu[(H - 1) * d + j] = 0.0;
}

/* ------------------------------------------------------------------------- */
/* One control step of Algorithm 1: shift (skipped at step 0), K iterations   */
/* of sample_controls / generate_rollouts / update_distribution, then         */
/* next_command = the first action of the mean.  Returns the OR of update     */
/* statuses (1 = degenerate: all costs non-finite).                            */
/* ------------------------------------------------------------------------- */
int orc_step(const orc_robot* R, const orc_world* W, const orc_params* P,
             const double* state, const double* goal, uint32_t step, double* mu,
             double* sigma, double* cmd, double* best_cost)
{
    const int N = P->N, H = P->H, d = R->dof;
    const int S = noise_samples(P);
    const long long count = (long long)N * S * d;
    double* eps = (double*)malloc(sizeof(double) * (size_t)count);
    double* u = (double*)malloc(sizeof(double) * (size_t)N * H * d);
    double* C = (double*)malloc(sizeof(double) * N);
    int status = 0;
    if (step > 0) orc_shift(H, d, mu);
    if (P->sampler == ORC_SAMPLER_HALTON) orc_noise_halton_ex(N, S, d, P->halton_scramble, P->seed, eps);
    for (int k = 0; k < P->K; ++k) {
        if (P->sampler == ORC_SAMPLER_PHILOX)
            orc_noise_philox(P->seed, step, P->instance, (uint32_t)k, 0u, count, eps);
        if (orc_rollout(R, W, P, state, goal, mu, sigma, eps, u, NULL, NULL, NULL, NULL, NULL, C))
            status |= 2;
        status |= orc_update(P, d, C, u, mu, sigma, NULL);
        if (best_cost) {
            double m = INFINITY;
            for (int n = 0; n < N; ++n)
                if (C[n] < m) m = C[n];
            *best_cost = m;
        }
    }
    /* optional gradient refinement: noise of iteration K + g, mu -= eta dJ/dmu */
    for (int g = 0; g < P->grad_steps; ++g) {
        double* grad = (double*)malloc(sizeof(double) * H * d);
        double J;
        if (P->sampler == ORC_SAMPLER_PHILOX)
            orc_noise_philox(P->seed, step, P->instance, (uint32_t)(P->K + g), 0u, count, eps);
        orc_cost_grad(R, W, P, state, goal, mu, sigma, eps, grad, &J, NULL);
        for (int k = 0; k < H * d; ++k) mu[k] -= P->grad_eta * grad[k];
        free(grad);
    }
    for (int j = 0; j < d; ++j) cmd[j] = mu[j];
    free(eps);
    free(u);
    free(C);
    return status;
}

/* ========================================================================= */
/* Adjoint of the rollout cost with respect to the mean control sequence.    */
/* The paper optimises the mean by sampling only; this gradient is an added  */
/* capability.  J(mu) = (1/N) sum_n C_n(u_n), u_n = mu + sigma o eps~_n with */
/* the noise fixed, so dJ/dmu = (1/N) sum_{n >= n_null} dC_n/du_n.  Every    */
/* derivative below is the hand-derived derivative of the forward routine   */
/* above; kinks take the zero subgradient (a norm at 0, a hinge at 0), the   */
/* min over collision pairs follows its first minimiser, and the            */
/* manipulability indicator is differentiated only where m < k_m.  Pinned by */
/* FP64 central finite differences away from kinks and by the explicit       */
/* transpose of the integration matrices.                                    */
/* ========================================================================= */

static void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* vee part of tr(A [w]x): returns v with tr(A [w]x) = v . w */
static void trace_skew(const double* A, double* v)
{
    v[0] = A[1 * 3 + 2] - A[2 * 3 + 1];
    v[1] = A[2 * 3 + 0] - A[0 * 3 + 2];
    v[2] = A[0 * 3 + 1] - A[1 * 3 + 0];
}

/* Inverse of an n x n matrix by Gauss-Jordan with partial pivoting; 0 if singular. */
static int invert(int n, const double* A, double* Ainv)
{
    double M[6 * 12];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c)
            M[r * 2 * n + c] = (c < n) ? A[r * n + c] : ((c - n == r) ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(M[r * 2 * n + c]) > fabs(M[piv * 2 * n + c])) piv = r;
        if (M[piv * 2 * n + c] == 0.0) return 0;
        for (int k = 0; k < 2 * n; ++k) {
            const double t = M[c * 2 * n + k];
            M[c * 2 * n + k] = M[piv * 2 * n + k];
            M[piv * 2 * n + k] = t;
        }
        const double inv = 1.0 / M[c * 2 * n + c];
        for (int k = 0; k < 2 * n; ++k) M[c * 2 * n + k] *= inv;
        for (int r = 0; r < n; ++r)
            if (r != c) {
                const double f = M[r * 2 * n + c];
                for (int k = 0; k < 2 * n; ++k) M[r * 2 * n + k] -= f * M[c * 2 * n + k];
            }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ainv[r * n + c] = M[r * 2 * n + n + c];
    return 1;
}

/* Add w * (dphi/dc)^T (dc/dtheta) for a point c rigidly attached to frame f:
 * dc/dtheta_k = z_k x (c - o_k) for joints k = 1..f. */
static void add_point_grad(const double* frames, int f, const double* c, const double* dphi_dc,
                           double w, double* g_theta)
{
    for (int k = 1; k <= f; ++k) {
        const double* T = frames + k * 16;
        const double z[3] = {T[2], T[6], T[10]};
        const double r[3] = {c[0] - T[3], c[1] - T[7], c[2] - T[11]};
        double v[3];
        cross3(z, r, v);
        g_theta[k - 1] += w * (dphi_dc[0] * v[0] + dphi_dc[1] * v[1] + dphi_dc[2] * v[2]);
    }
}

/* Gradient of the running cost c_hat_h (Eq. 15) with respect to theta_h,
 * theta_dot_h, u_h and u_{h-1}. */
void orc_running_cost_grad(const orc_robot* R, const orc_world* W, const orc_params* P,
                           const double* goal, int h, const double* theta_h,
                           const double* theta_dot_h, const double* u_h, const double* u_prev,
                           double* g_th, double* g_thd, double* g_u, double* g_up)
{
    const int d = R->dof, H = P->H;
    double* frames = (double*)malloc(sizeof(double) * 16 * (d + 1));
    double J[6 * 8];
    orc_fk(R, theta_h, frames);
    orc_jacobian(R, frames, J);
    for (int j = 0; j < d; ++j) g_th[j] = g_thd[j] = g_u[j] = g_up[j] = 0.0;
    const double* Te = frames + d * 16;
    const double Ree[9] = {Te[0], Te[1], Te[2], Te[4], Te[5], Te[6], Te[8], Te[9], Te[10]};
    double Rg[9];
    orc_rot_from_quat(goal + 3, Rg);

    /* position (Eq. 9): d||e||/dp = R_g (alpha_2 o e) / ||e||, then J_v^T */
    {
        const double dp[3] = {Te[3] - goal[0], Te[7] - goal[1], Te[11] - goal[2]};
        double e[3], c = 0.0;
        for (int i = 0; i < 3; ++i) {
            e[i] = P->pos_axis_w[i] *
                   (Rg[0 * 3 + i] * dp[0] + Rg[1 * 3 + i] * dp[1] + Rg[2 * 3 + i] * dp[2]);
            c += e[i] * e[i];
        }
        c = sqrt(c);
        if (c > 0.0) {
            double gp[3];
            for (int r = 0; r < 3; ++r) {
                gp[r] = 0.0;
                for (int i = 0; i < 3; ++i) gp[r] += Rg[r * 3 + i] * P->pos_axis_w[i] * e[i] / c;
            }
            for (int k = 0; k < d; ++k)
                g_th[k] += P->w_pos * (gp[0] * J[0 * d + k] + gp[1] * J[1 * d + k] + gp[2] * J[2 * d + k]);
        }
    }
    /* rotation (Eq. 9): dR = [w]x R with w = J_w dtheta */
    {
        double gw[3] = {0.0, 0.0, 0.0};
        if (P->rot_mode == ORC_ROT_QUAT) {
            /* 1 - |q_ee . q_g| = 1 - sqrt(1 + tr(R_g^T R_ee)) / 2 */
            double tr = 0.0;
            for (int k = 0; k < 9; ++k) tr += Rg[k] * Ree[k];
            if (1.0 + tr > 0.0) {
                double A[9], v[3]; /* A = R_ee R_g^T */
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c) {
                        A[r * 3 + c] = 0.0;
                        for (int k = 0; k < 3; ++k) A[r * 3 + c] += Ree[r * 3 + k] * Rg[c * 3 + k];
                    }
                trace_skew(A, v);
                const double dc_dtr = -0.25 / sqrt(1.0 + tr);
                for (int i = 0; i < 3; ++i) gw[i] = dc_dtr * v[i];
            }
        } else {
            double E[9], c = 0.0;
            for (int r = 0; r < 3; ++r)
                for (int q = 0; q < 3; ++q) {
                    double RtR = 0.0;
                    for (int k = 0; k < 3; ++k) RtR += Rg[k * 3 + r] * Ree[k * 3 + q];
                    E[r * 3 + q] = ((r == q) ? 1.0 : 0.0) - RtR;
                    c += (E[r * 3 + q] * P->rot_axis_w[q]) * (E[r * 3 + q] * P->rot_axis_w[q]);
                }
            c = sqrt(c);
            if (c > 0.0) {
                /* dc = (1/c) tr(M^T dE), M = E diag(alpha_1^2), dE = -R_g^T [w]x R_ee
                 *    = -(1/c) tr(A [w]x) with A = R_ee M^T R_g^T */
                double Mt[9], A[9], tmp[9], v[3];
                for (int r = 0; r < 3; ++r)
                    for (int q = 0; q < 3; ++q)
                        Mt[q * 3 + r] = E[r * 3 + q] * P->rot_axis_w[q] * P->rot_axis_w[q];
                for (int r = 0; r < 3; ++r)
                    for (int q = 0; q < 3; ++q) {
                        tmp[r * 3 + q] = 0.0;
                        for (int k = 0; k < 3; ++k) tmp[r * 3 + q] += Ree[r * 3 + k] * Mt[k * 3 + q];
                    }
                for (int r = 0; r < 3; ++r)
                    for (int q = 0; q < 3; ++q) {
                        A[r * 3 + q] = 0.0;
                        for (int k = 0; k < 3; ++k) A[r * 3 + q] += tmp[r * 3 + k] * Rg[q * 3 + k];
                    }
                trace_skew(A, v);
                for (int i = 0; i < 3; ++i) gw[i] = -v[i] / c;
            }
        }
        for (int k = 0; k < d; ++k)
            g_th[k] += P->w_rot * (gw[0] * J[3 * d + k] + gw[1] * J[4 * d + k] + gw[2] * J[5 * d + k]);
    }
    /* stop (Eq. 10), joint limits (Eq. 11), smoothness */
    {
        double vmax = 0.0;
        for (int k = 0; k < H; ++k) vmax += (k >= h ? 1.0 : 0.0) * P->qdd_max * P->dt[k];
        double vs[8], vj[8], cs = 0.0, cj = 0.0;
        for (int j = 0; j < d; ++j) {
            vs[j] = fabs(theta_dot_h[j]) - vmax;
            if (vs[j] < 0.0) vs[j] = 0.0;
            cs += vs[j] * vs[j];
            const double range = R->q_max[j] - R->q_min[j];
            const double lo = R->q_min[j] + P->k_jl * range, hi = R->q_max[j] - P->k_jl * range;
            vj[j] = (theta_h[j] < lo ? lo - theta_h[j] : 0.0) + (theta_h[j] > hi ? theta_h[j] - hi : 0.0);
            cj += vj[j] * vj[j];
            const double du = u_h[j] - u_prev[j];
            g_u[j] += P->w_smooth * 2.0 * du;
            g_up[j] -= P->w_smooth * 2.0 * du;
        }
        cs = sqrt(cs);
        cj = sqrt(cj);
        for (int j = 0; j < d; ++j) {
            if (cs > 0.0 && vs[j] > 0.0)
                g_thd[j] += P->w_stop * vs[j] * (theta_dot_h[j] > 0.0 ? 1.0 : -1.0) / cs;
            if (cj > 0.0 && vj[j] > 0.0) {
                const double range = R->q_max[j] - R->q_min[j];
                const double lo = R->q_min[j] + P->k_jl * range;
                g_th[j] += P->w_joint * vj[j] * (theta_h[j] < lo ? -1.0 : 1.0) / cj;
            }
        }
    }
    /* manipulability (Eq. 12): dm/dtheta_k = m tr(J0^+ dJ0/dtheta_k), with J0 the
     * geometric Jacobian about the base origin (same det(J J^T)), columns
     * [o_i x z_i; z_i]; dz_i/dtheta_k = z_k x z_i and do_i/dtheta_k =
     * z_k x (o_i - o_k) for k < i, zero otherwise. */
    {
        const double m = orc_manipulability(J, d);
        if (m < P->k_m && m > 0.0 && P->w_manip != 0.0) {
            double z[8][3], o[8][3], J0[6 * 8], G[36], Gi[36];
            for (int i = 0; i < d; ++i) {
                const double* T = frames + (i + 1) * 16;
                z[i][0] = T[2], z[i][1] = T[6], z[i][2] = T[10];
                o[i][0] = T[3], o[i][1] = T[7], o[i][2] = T[11];
                double oz[3];
                cross3(o[i], z[i], oz);
                for (int r = 0; r < 3; ++r) {
                    J0[r * d + i] = oz[r];
                    J0[(3 + r) * d + i] = z[i][r];
                }
            }
            for (int r = 0; r < 6; ++r)
                for (int c = 0; c < 6; ++c) {
                    G[r * 6 + c] = 0.0;
                    for (int k = 0; k < d; ++k) G[r * 6 + c] += J0[r * d + k] * J0[c * d + k];
                }
            if (invert(6, G, Gi)) {
                double Jp[8 * 6]; /* J0^T G^-1, d x 6 */
                for (int i = 0; i < d; ++i)
                    for (int r = 0; r < 6; ++r) {
                        Jp[i * 6 + r] = 0.0;
                        for (int k = 0; k < 6; ++k) Jp[i * 6 + r] += J0[k * d + i] * Gi[k * 6 + r];
                    }
                for (int k = 0; k < d; ++k) {
                    double tr = 0.0;
                    for (int i = k + 1; i < d; ++i) {
                        double dz[3], doo[3], rel[3], a[3], b[3];
                        cross3(z[k], z[i], dz);
                        for (int q = 0; q < 3; ++q) rel[q] = o[i][q] - o[k][q];
                        cross3(z[k], rel, doo);
                        cross3(doo, z[i], a);
                        cross3(o[i], dz, b);
                        for (int q = 0; q < 3; ++q) {
                            tr += Jp[i * 6 + q] * (a[q] + b[q]);
                            tr += Jp[i * 6 + 3 + q] * dz[q];
                        }
                    }
                    g_th[k] += P->w_manip * (-m * tr);
                }
            }
        }
    }
    /* self collision (Eq. 13 reading): first minimising pair */
    if (P->w_coll != 0.0) {
        double best = INFINITY, na[3] = {0, 0, 0}, ca_b[3], cb_b[3];
        int ba = -1, bb = -1;
        for (int k = 0; k < R->n_pairs; ++k) {
            const int a = R->pairs[2 * k], b = R->pairs[2 * k + 1];
            double ca[3], cb[3];
            sphere_center(R, frames, a, ca);
            sphere_center(R, frames, b, cb);
            const double dist = sqrt((ca[0] - cb[0]) * (ca[0] - cb[0]) + (ca[1] - cb[1]) * (ca[1] - cb[1]) +
                                     (ca[2] - cb[2]) * (ca[2] - cb[2]));
            const double sd = dist - R->sphere[a * 4 + 3] - R->sphere[b * 4 + 3];
            if (sd < best) {
                best = sd;
                ba = a;
                bb = b;
                for (int q = 0; q < 3; ++q) {
                    na[q] = dist > 0.0 ? (ca[q] - cb[q]) / dist : 0.0;
                    ca_b[q] = ca[q];
                    cb_b[q] = cb[q];
                }
            }
        }
        if (ba >= 0 && best < 0.0) {
            /* c_self = -sd: d(-sd)/dc_a = -n, d(-sd)/dc_b = +n */
            const double mn[3] = {-na[0], -na[1], -na[2]};
            add_point_grad(frames, R->sphere_link[ba], ca_b, mn, P->w_coll, g_th);
            add_point_grad(frames, R->sphere_link[bb], cb_b, na, P->w_coll, g_th);
        }
    }
    /* world collision (Eq. 14 reading): first minimising (sphere, obstacle) */
    if (P->w_coll != 0.0) {
        double best = INFINITY, grad_c[3] = {0, 0, 0}, cbest[3];
        int bs = -1;
        for (int s = 0; s < R->n_spheres; ++s) {
            double c[3];
            sphere_center(R, frames, s, c);
            const double r = R->sphere[s * 4 + 3];
            for (int b = 0; b < W->n_boxes; ++b) {
                const double* box = W->boxes + b * 6;
                const double sd = orc_box_sdf(c, box) - r;
                if (sd < best) {
                    best = sd;
                    bs = s;
                    memcpy(cbest, c, sizeof(cbest));
                    double q[3], out = 0.0;
                    int kmax = 0;
                    for (int k = 0; k < 3; ++k) {
                        q[k] = fabs(c[k] - box[k]) - box[3 + k];
                        if (q[k] > 0.0) out += q[k] * q[k];
                        if (q[k] > q[kmax]) kmax = k;
                    }
                    out = sqrt(out);
                    for (int k = 0; k < 3; ++k) {
                        const double sgn = (c[k] - box[k]) >= 0.0 ? 1.0 : -1.0;
                        if (out > 0.0)
                            grad_c[k] = q[k] > 0.0 ? sgn * q[k] / out : 0.0;
                        else
                            grad_c[k] = (k == kmax) ? sgn : 0.0;
                    }
                }
            }
            for (int o = 0; o < W->n_spheres; ++o) {
                const double* S = W->spheres + o * 4;
                const double dist = sqrt((c[0] - S[0]) * (c[0] - S[0]) + (c[1] - S[1]) * (c[1] - S[1]) +
                                         (c[2] - S[2]) * (c[2] - S[2]));
                const double sd = dist - r - S[3];
                if (sd < best) {
                    best = sd;
                    bs = s;
                    memcpy(cbest, c, sizeof(cbest));
                    for (int k = 0; k < 3; ++k) grad_c[k] = dist > 0.0 ? (c[k] - S[k]) / dist : 0.0;
                }
            }
        }
        if (bs >= 0 && best < 0.0) {
            const double mg[3] = {-grad_c[0], -grad_c[1], -grad_c[2]};
            add_point_grad(frames, R->sphere_link[bs], cbest, mg, P->w_coll, g_th);
        }
    }
    free(frames);
}

/* Adjoint of the integration (Eq. 7) for one particle: given G_theta_h,
 * G_theta_dot_h, G_u_h (all H x d, already discounted), returns dC/du_k =
 * G_u_k + dt_k sum_{h>=k} (G_theta_dot_h + dt_h sum_{m>=h} G_theta_m), i.e.
 * the transposes of the inclusive lower-triangular S_l(1) diag(dt) products. */
void orc_integrate_adjoint(int H, int d, const double* dt, const double* g_th, const double* g_thd,
                           const double* g_u, double* dC_du)
{
    for (int j = 0; j < d; ++j) {
        for (int k = 0; k < H; ++k) {
            /* total derivative with respect to theta_dot_k */
            double acc = 0.0;
            for (int h = k; h < H; ++h) {
                double tv = g_thd[h * d + j];
                for (int m = h; m < H; ++m) tv += dt[h] * g_th[m * d + j];
                acc += tv;
            }
            dC_du[k * d + j] = g_u[k * d + j] + dt[k] * acc;
        }
    }
}

int orc_cost_grad(const orc_robot* R, const orc_world* W, const orc_params* P,
                  const double* state, const double* goal, const double* mu, const double* sigma,
                  const double* eps, double* grad_mu, double* Jval, double* dC_du_out)
{
    const int N = P->N, H = P->H, d = R->dof;
    if (N <= 0 || H <= 0 || d <= 0 || d > 8) return -1;
    /* the adjoint covers the paper's cost terms and the default smoothing */
    if (P->filter != ORC_FILTER_DEFAULT || P->w_ee_vel != 0.0 || P->w_ee_acc != 0.0 || P->w_ball != 0.0)
        return -2;
    double* u = (double*)malloc(sizeof(double) * (size_t)N * H * d);
    double* th = (double*)malloc(sizeof(double) * H * d);
    double* thd = (double*)malloc(sizeof(double) * H * d);
    double* Gth = (double*)malloc(sizeof(double) * H * d);
    double* Gthd = (double*)malloc(sizeof(double) * H * d);
    double* Gu = (double*)malloc(sizeof(double) * H * d);
    double* dCdu = (double*)malloc(sizeof(double) * H * d);
    orc_smooth_controls(P, d, mu, sigma, eps, u);
    for (int k = 0; k < H * d; ++k) grad_mu[k] = 0.0;
    double Jacc = 0.0;
    for (int n = 0; n < N; ++n) {
        const double* un = u + (size_t)n * H * d;
        orc_integrate(H, d, P->dt, state, un, th, thd);
        for (int k = 0; k < H * d; ++k) Gth[k] = Gthd[k] = Gu[k] = 0.0;
        double C = 0.0;
        for (int h = 0; h < H; ++h) {
            double terms[ORC_NTERMS], c, gt[8], gtd[8], gu[8], gup[8];
            const double* uprev = (h == 0) ? state + 2 * d : un + (h - 1) * d;
            orc_running_cost(R, W, P, goal, h, th + h * d, thd + h * d, un + h * d, uprev, terms, &c);
            const double gam = pow(P->gamma, (double)h);
            C += gam * c;
            orc_running_cost_grad(R, W, P, goal, h, th + h * d, thd + h * d, un + h * d, uprev, gt,
                                  gtd, gu, gup);
            for (int j = 0; j < d; ++j) {
                Gth[h * d + j] += gam * gt[j];
                Gthd[h * d + j] += gam * gtd[j];
                Gu[h * d + j] += gam * gu[j];
                if (h > 0) Gu[(h - 1) * d + j] += gam * gup[j];
            }
        }
        Jacc += C;
        orc_integrate_adjoint(H, d, P->dt, Gth, Gthd, Gu, dCdu);
        if (dC_du_out) memcpy(dC_du_out + (size_t)n * H * d, dCdu, sizeof(double) * H * d);
        if (n >= P->n_null)
            for (int k = 0; k < H * d; ++k) grad_mu[k] += dCdu[k] / N;
    }
    *Jval = Jacc / N;
    free(u);
    free(th);
    free(thd);
    free(Gth);
    free(Gthd);
    free(Gu);
    free(dCdu);
    return 0;
}

/* ========================================================================= */
/* Self-collision surrogate network.  The paper learns the closest distance  */
/* between links with an MLP (Sec. 4.2, Eq. 13); this is the network of the */
/* surrogate workload: encoded joints -> 256 -> 256 -> 256 -> 1 with ReLU.   */
/* Encoding: x_j = theta_j / 3 (j < dof), x_7 = 1 (so the first layer's      */
/* bias is its weight column 7), other inputs 0 (16 inputs).                 */
/* Flat parameters (row-major, out x in): W1 256x16 | W2 256x256 | b2 256 |   */
/* W3 256x256 | b3 256 | w4 256 | b4 1.                                      */
/* With bf16 != 0 the routine rounds, exactly where a BF16 tensor-core      */
/* implementation stores an operand, to the nearest BF16 (ties to even):    */
/* W1..W3, the inputs, the hidden activations a1, a2, a3 and the back-      */
/* propagated deltas; sums stay in double.  Pinned by finite differences    */
/* (bf16 = 0) and a hand-computed tiny network.                              */
/* ========================================================================= */

#define H_ ORC_MLP_HID
#define I_ ORC_MLP_IN

/* Surrogate networks for the self-collision term (Sec. 4.2, Eq. 13).  Layers:
 * x (16) -> h1 -> h2 -> h3 -> 1, ReLU on the hidden layers, no bias on the
 * first (the encoding carries a constant-one feature), a linear output.
 * Parameters flat: W1 (h1 x 16) | W2 (h2 x h1) | b2 | W3 (h3 x h2) | b3 |
 * w4 (h3) | b4.  Encodings: SCALED x_j = theta_j / 3, x_7 = 1 (the 256-256-256
 * distance network); SINCOS x_j = sin theta_j, x_{7+j} = cos theta_j, x_14 = 1
 * (jointNERF's positional encoding, hidden [256, 128, 64]). */
static const orc_mlp_arch k_arch_default = {ORC_ENC_SCALED, 256, 256, 256};

long orc_mlp_arch_param_count(const orc_mlp_arch* A)
{
    return (long)A->h1 * I_ + (long)A->h2 * A->h1 + A->h2 + (long)A->h3 * A->h2 + A->h3 + A->h3 + 1;
}

long orc_mlp_param_count(void) { return orc_mlp_arch_param_count(&k_arch_default); }

/* Round to the nearest bfloat16 (ties to even) through binary32. */
float orc_bf16_round(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x; /* inf / nan unchanged */
    const uint32_t lsb = (u >> 16) & 1u;
    u = (u + 0x7fffu + lsb) & 0xffff0000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

static double q(double v, int bf16) { return bf16 ? (double)orc_bf16_round((float)v) : v; }

void orc_mlp_arch_encode(const orc_mlp_arch* A, const double* theta, int dof, double* x)
{
    for (int i = 0; i < I_; ++i) x[i] = 0.0;
    if (A->enc == ORC_ENC_SINCOS) {
        for (int j = 0; j < dof && j < 7; ++j) {
            x[j] = sin(theta[j]);
            x[7 + j] = cos(theta[j]);
        }
        x[14] = 1.0;
    } else {
        for (int j = 0; j < dof && j < 7; ++j) x[j] = theta[j] / 3.0;
        x[7] = 1.0;
    }
}

void orc_mlp_encode(const double* theta, int dof, double* x) { orc_mlp_arch_encode(&k_arch_default, theta, dof, x); }

typedef struct {
    const double *W1, *W2, *b2, *W3, *b3, *w4, *b4;
} mlp_view;

static mlp_view mlp_split(const orc_mlp_arch* A, const double* p)
{
    mlp_view v;
    v.W1 = p;
    v.W2 = v.W1 + A->h1 * I_;
    v.b2 = v.W2 + A->h2 * A->h1;
    v.W3 = v.b2 + A->h2;
    v.b3 = v.W3 + A->h3 * A->h2;
    v.w4 = v.b3 + A->h3;
    v.b4 = v.w4 + A->h3;
    return v;
}

/* one sample: activations a1 (h1), a2 (h2), a3 (h3) and output; with bf16 the
 * operands of the three GEMM layers are rounded as the tensor-core path rounds
 * them (inputs, weights, a1, a2), the output layer reads the unrounded a3 */
static double mlp_one(const orc_mlp_arch* A, const mlp_view* v, const double* x_in, int bf16, double* a1,
                      double* a2, double* a3)
{
    double x[I_];
    for (int i = 0; i < I_; ++i) x[i] = q(x_in[i], bf16);
    for (int n = 0; n < A->h1; ++n) {
        double z = 0.0;
        for (int k = 0; k < I_; ++k) z += q(v->W1[n * I_ + k], bf16) * x[k];
        a1[n] = q(z > 0.0 ? z : 0.0, bf16);
    }
    for (int n = 0; n < A->h2; ++n) {
        double z = 0.0;
        for (int k = 0; k < A->h1; ++k) z += q(v->W2[n * A->h1 + k], bf16) * a1[k];
        z += v->b2[n];
        a2[n] = q(z > 0.0 ? z : 0.0, bf16);
    }
    double y = v->b4[0];
    for (int n = 0; n < A->h3; ++n) {
        double z = 0.0;
        for (int k = 0; k < A->h2; ++k) z += q(v->W3[n * A->h2 + k], bf16) * a2[k];
        z += v->b3[n];
        const double a = z > 0.0 ? z : 0.0;
        y += v->w4[n] * a;
        a3[n] = q(a, bf16);
    }
    return y;
}

enum { MAXH_ = 256 };

void orc_mlp_arch_forward(const orc_mlp_arch* A, const double* params, const double* theta, int B, int dof,
                          int bf16, double* y)
{
    const mlp_view v = mlp_split(A, params);
    double x[I_], a1[MAXH_], a2[MAXH_], a3[MAXH_];
    for (int b = 0; b < B; ++b) {
        orc_mlp_arch_encode(A, theta + b * dof, dof, x);
        y[b] = mlp_one(A, &v, x, bf16, a1, a2, a3);
    }
}

void orc_mlp_forward(const double* params, const double* theta, int B, int dof, int bf16, double* y)
{
    orc_mlp_arch_forward(&k_arch_default, params, theta, B, dof, bf16, y);
}

/* Mean squared error (1/B) sum (y_b - t_b)^2 and its gradient, by the chain
 * rule written layer by layer (delta_l = (W_{l+1}^T delta_{l+1}) o [z_l > 0]). */
double orc_mlp_arch_loss_grad(const orc_mlp_arch* A, const double* params, const double* theta,
                              const double* target, int B, int dof, int bf16, double* grad)
{
    const int h1 = A->h1, h2 = A->h2, h3 = A->h3;
    const mlp_view v = mlp_split(A, params);
    const long P = orc_mlp_arch_param_count(A);
    for (long i = 0; i < P; ++i) grad[i] = 0.0;
    double* gW1 = grad;
    double* gW2 = gW1 + h1 * I_;
    double* gb2 = gW2 + h2 * h1;
    double* gW3 = gb2 + h2;
    double* gb3 = gW3 + h3 * h2;
    double* gw4 = gb3 + h3;
    double* gb4 = gw4 + h3;
    double loss = 0.0;
    double x[I_], xq[I_], a1[MAXH_], a2[MAXH_], a3[MAXH_], d3[MAXH_], d2[MAXH_], d1[MAXH_];
    for (int b = 0; b < B; ++b) {
        orc_mlp_arch_encode(A, theta + b * dof, dof, x);
        const double y = mlp_one(A, &v, x, bf16, a1, a2, a3);
        for (int i = 0; i < I_; ++i) xq[i] = q(x[i], bf16);
        const double r = y - target[b];
        loss += r * r / B;
        const double dy = 2.0 * r / B;
        gb4[0] += dy;
        for (int n = 0; n < h3; ++n) {
            gw4[n] += dy * a3[n];
            d3[n] = q(a3[n] > 0.0 ? dy * v.w4[n] : 0.0, bf16);
        }
        for (int n = 0; n < h3; ++n) {
            gb3[n] += d3[n];
            for (int k = 0; k < h2; ++k) gW3[n * h2 + k] += d3[n] * a2[k];
        }
        for (int k = 0; k < h2; ++k) {
            double s = 0.0;
            for (int n = 0; n < h3; ++n) s += d3[n] * q(v.W3[n * h2 + k], bf16);
            d2[k] = q(a2[k] > 0.0 ? s : 0.0, bf16);
        }
        for (int n = 0; n < h2; ++n) {
            gb2[n] += d2[n];
            for (int k = 0; k < h1; ++k) gW2[n * h1 + k] += d2[n] * a1[k];
        }
        for (int k = 0; k < h1; ++k) {
            double s = 0.0;
            for (int n = 0; n < h2; ++n) s += d2[n] * q(v.W2[n * h1 + k], bf16);
            d1[k] = q(a1[k] > 0.0 ? s : 0.0, bf16);
        }
        for (int n = 0; n < h1; ++n)
            for (int k = 0; k < I_; ++k) gW1[n * I_ + k] += d1[n] * xq[k];
    }
    return loss;
}

double orc_mlp_loss_grad(const double* params, const double* theta, const double* target, int B, int dof,
                         int bf16, double* grad)
{
    return orc_mlp_arch_loss_grad(&k_arch_default, params, theta, target, B, dof, bf16, grad);
}

/* Exact label of the surrogate: the minimum signed distance over the self
 * pairs (positive apart) for one configuration. */
double orc_self_min_sd_theta(const orc_robot* R, const double* theta)
{
    double* frames = (double*)malloc(sizeof(double) * 16 * (R->dof + 1));
    orc_fk(R, theta, frames);
    const double sd = orc_self_min_sd(R, frames);
    free(frames);
    return sd;
}
#undef H_
#undef I_
