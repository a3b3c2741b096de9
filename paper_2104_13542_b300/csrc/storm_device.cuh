// storm_device.cuh -- device-side building blocks of the STORM control step.
//
// Counter-based noise (Philox4x32-10 + Box-Muller), the modified-DH chain
// step, the manipulability score and the per-problem parameter block that
// every kernel receives by value.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "storm.h"

namespace storm {

constexpr int kMaxDof = 7;
constexpr int kThreads = 256;        // default rollout CTA size
constexpr int kMaxThreads = 512;     // largest rollout CTA size the tuner may pick
constexpr int kUpdateThreads = 512;  // distribution-update CTA size (one CTA per horizon step)
constexpr int kLinkPairs = (kMaxDof + 1) * kMaxDof / 2;  // frame pairs (la < lb) of a chain
constexpr int kMlpRows = 128;       // rows of a tensor-core tile of the self-collision network

// Position of frame pair (la, lb), la < lb <= kMaxDof, in lexicographic order.
__host__ __device__ constexpr int link_pair_index(int la, int lb)
{
    return la * kMaxDof - la * (la - 1) / 2 + (lb - la - 1);
}

// Per-problem constants and device table pointers (kernel parameter, by value).
struct Problem {
    int N, H, d, S;          // particles, horizon, joints, noise knots (S = H without spline)
    int spline;              // 1 when the noise is smoothed by the B-spline basis
    int sampler, n_null, rot_mode;
    int M, P, B, O;          // link spheres, self pairs, boxes, obstacle spheres
    int ppc;                 // particles per rollout CTA
    float beta, alpha_mu, alpha_sigma, sigma_min;
    float w_pos, w_rot, w_stop, w_joint, w_manip, w_coll, w_smooth;
    float pos_w[3], rot_w[3];
    float k_m;
    uint32_t seed_lo, seed_hi, instance;
    const float* dhx;        // d x 8: a, cos alpha, sin alpha, d, offset, -, -, -
    const float* qlo;        // d soft lower limits  q_min + k_jl (q_max - q_min)
    const float* qhi;        // d soft upper limits  q_max - k_jl (q_max - q_min)
    const float4* sph;       // M: centre in link frame, radius (sorted by link)
    const int* link_first;   // d + 2: spheres of frame f are [link_first[f], link_first[f+1])
    const uint32_t* pairs;   // P: a | b << 16 (sorted sphere indices), pairs outside blocks
    int NPB;                 // pair blocks
    const uint4* pblk;       // NPB: (a0, a1, b0, nb): spheres [a0, a1) x [b0, b0 + nb), nb <= 8
    const float4* lbound;    // d + 1: bounding sphere of each frame's spheres (local centre, radius)
    const float4* lcap;      // 2 (d + 1): capsule of each frame's spheres, local: (end 0, radius), (end 1, 0)
    int broadphase;          // 1: exact sphere tests only where the link bounds overlap
    int dep_launch;          // 1: this rollout launch is a programmatic dependent
    int shift_view;          // 1: read mu shifted (row h = stored row h + 1, last row 0) once the
                             // step counter is > 0 -- the first rollout of a step (Alg. 1's shift)
    unsigned long long* trace;  // nullable: phase-boundary %globaltimer stamps of rollout CTA 0
    const uint4* tables;     // start of the contiguous per-problem tables (dhx .. basis)
    int table_bytes;         // their size, a multiple of 16
    const float* boxes;      // B x 6
    const float4* wsph;      // O
    const float* dt;         // H
    const float* gpow;       // H: gamma^h
    const float* vmax;       // H: qdd_max * sum_{k >= h} dt_k
    const float* basis;      // H x S B-spline basis (spline only)
    const float* halton;     // N x S x d normal noise (Halton sampler only)
    float* mu;               // H x d
    float* sigma;            // d
    // learned self collision (Sec. 4.2), evaluated inside the rollout kernel: 0 the exact
    // check; 1 the exact check only where the network's predicted distance is below
    // self_margin (elsewhere the self term is 0); 2 the self term is max(0, network), the
    // network predicting the penetration depth (Eq. 13), no exact check
    int self_mode;
    float self_margin;
    // pair blocks of frames (la, lb), la < lb, are [lp_begin[t], lp_begin[t + 1]) with
    // t = link_pair_index(la, lb); the blocks are sorted by (la, lb)
    uint16_t lp_begin[kLinkPairs + 1];
    // noise smoothing (Sec. 4.3)
    int filter;              // STORM_FILTER_*
    int nk;                  // B-spline knots (basis columns); the basis is H x nk
    int n_bs;                // mixed filter: particles [n_null, n_null + n_bs) take the B-spline
    float comb[3];           // comb-filter coefficients
    // task-space limits on the end-effector speed and acceleration (Eq. 8)
    float w_ee_vel, w_ee_acc, ee_vel_max, ee_acc_max;
    // ball on a tray
    float w_ball, grav[3], tray[3];
    const float* ball;       // 6: ball position, velocity (world frame); nullable: no ball
};

// Step bookkeeping kept on the device so captured graphs need no host update.
struct StepState {
    uint32_t step;   // index of the next control step
    int status;      // OR of warnings of the current step
    float best;      // min total cost of the last iteration
    float wmean;     // weighted mean total cost of the last iteration
};

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialisation may start while its predecessor in the stream still runs:
// pdl_wait blocks until that predecessor has completed and its writes are
// visible to this grid; pdl_trigger lets this kernel's own dependent start
// launching its CTAs.  Both are no-ops for a kernel launched the ordinary way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Phase stamp of the rollout trace (CTA 0, thread 0 only).
__device__ __forceinline__ void trace_stamp(unsigned long long* trace, int phase)
{
    if (trace && blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        trace[phase] = t;
    }
}

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., SC'11: ten rounds of two 32x32->64 multiplies with a Weyl key
// schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// 23 high bits, centred: exactly representable in float, strictly inside (0, 1).
__device__ __forceinline__ float bits_to_unit(uint32_t x)
{
    return (static_cast<float>(x >> 9) + 0.5f) * (1.0f / 8388608.0f);
}

// Box-Muller pair from two words.
__device__ __forceinline__ float2 gauss_pair(uint32_t a, uint32_t b)
{
    const float r = sqrtf(-2.0f * logf(bits_to_unit(a)));
    float s, c;
    sincospif(2.0f * bits_to_unit(b), &s, &c);
    return make_float2(r * c, r * s);
}

// ---------------------------------------------------------------- kinematics
// One modified-DH link: T <- T RotX(alpha) TransX(a) RotZ(theta) TransZ(d),
// with R row-major 3x3 and p the origin.  In place.
// sin and cos of a joint angle, branch-free: Cody-Waite reduction by pi/2
// (pi/2 split in three parts, the upper two with few enough significant bits
// that q times them is exact for |q| < 2^13, each step one FMA), then the
// Cephes single-precision minimax polynomials for sin and cos on
// [-pi/4, pi/4] (S. L. Moshier, Cephes Math Library, sinf.c / cosf.c), swapped
// and signed by the quadrant q mod 4.  Max error about 1e-7 absolute for
// |x| < 10^4; NaN and infinities give NaN.  The chain calls it once per joint
// of every (particle, step) item, so it is kept short and without a
// large-argument branch.
__device__ __forceinline__ void joint_sincos(float x, float& s, float& c)
{
    const float q = rintf(x * 0.636619772f);
    float r = fmaf(-q, 1.5703125f, x);
    r = fmaf(-q, 4.837512969970703125e-4f, r);
    r = fmaf(-q, 7.54978995489188216e-8f, r);
    const float z = r * r;
    const float sp = fmaf(fmaf(fmaf(-1.9515295891e-4f, z, 8.3321608736e-3f), z, -1.6666654611e-1f), z * r, r);
    const float cp = fmaf(fmaf(fmaf(2.443315711809948e-5f, z, -1.388731625493765e-3f), z, 4.166664568298827e-2f),
                          z * z, fmaf(-0.5f, z, 1.0f));
    const int k = static_cast<int>(q);
    // x = k pi/2 + r: (sin, cos) = (sp, cp), (cp, -sp), (-sp, -cp), (-cp, sp) for k mod 4 = 0..3
    const float s0 = (k & 1) ? cp : sp;
    const float c0 = (k & 1) ? sp : cp;
    s = (k & 2) ? -s0 : s0;
    c = ((k + 1) & 2) ? -c0 : c0;
}

__device__ __forceinline__ void dh_step(float (&R)[9], float (&p)[3], float a, float ca, float sa,
                                        float dd, float theta)
{
    float st, ct;
    joint_sincos(theta, st, ct);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float c0 = R[r * 3 + 0], c1 = R[r * 3 + 1], c2 = R[r * 3 + 2];
        const float x1 = fmaf(ca, c1, sa * c2);
        const float x2 = fmaf(-sa, c1, ca * c2);
        p[r] = fmaf(dd, x2, fmaf(a, c0, p[r]));
        R[r * 3 + 0] = fmaf(ct, c0, st * x1);
        R[r * 3 + 1] = fmaf(-st, c0, ct * x1);
        R[r * 3 + 2] = x2;
    }
}

// sqrt(det(J J^T)) of a 6 x d Jacobian given as rows, by modified Gram-Schmidt
// on the six rows: det(J J^T) is the product of the squared norms of the
// orthogonalised rows.  Six dependent reciprocal square roots; the dot
// products of one row against the earlier ones are independent.
__device__ __forceinline__ float manipulability_mgs(float (&J)[6][kMaxDof], int d)
{
    float m = 1.0f;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
#pragma unroll
        for (int i = 0; i < k; ++i) {
            float dot = 0.0f;
#pragma unroll
            for (int c = 0; c < kMaxDof; ++c)
                if (c < d) dot = fmaf(J[i][c], J[k][c], dot);
#pragma unroll
            for (int c = 0; c < kMaxDof; ++c)
                if (c < d) J[k][c] = fmaf(-dot, J[i][c], J[k][c]);
        }
        float nn = 0.0f;
#pragma unroll
        for (int c = 0; c < kMaxDof; ++c)
            if (c < d) nn = fmaf(J[k][c], J[k][c], nn);
        const float inv = nn > 0.0f ? rsqrtf(nn) : 0.0f;
        m *= nn * inv;  // the row's norm
#pragma unroll
        for (int c = 0; c < kMaxDof; ++c) J[k][c] *= inv;
    }
    return m;
}

// Manipulability sqrt(det(J J^T)) (Eq. 12) accumulated one Jacobian column at
// a time.  R is the upper-triangular 6x6 factor with R^T R = sum_i J_i J_i^T
// (21 packed entries, row-major upper triangle); adding column x is a
// rank-one update done with Givens rotations (the QR update of appending a
// row to the data matrix), which keeps the accuracy of an orthogonal
// factorisation.  Then det(J J^T) = prod R_kk^2.
struct GramFactor {
    float r[21];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int k = 0; k < 21; ++k) r[k] = 0.f;
    }
    // packed index of R[i][j], i <= j
    __device__ static constexpr int at(int i, int j) { return i * 6 - (i * (i - 1)) / 2 + (j - i); }
    __device__ __forceinline__ void add(float (&x)[6])
    {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float a = r[at(k, k)], b = x[k];
            const float hh = fmaf(a, a, b * b);
            const float inv = hh > 0.f ? rsqrtf(hh) : 0.f;
            const float c = hh > 0.f ? a * inv : 1.f, s = b * inv;
            r[at(k, k)] = hh * inv;  // sqrt(a^2 + b^2)
#pragma unroll
            for (int j = k + 1; j < 6; ++j) {
                const float rkj = r[at(k, j)], xj = x[j];
                r[at(k, j)] = fmaf(c, rkj, s * xj);
                x[j] = fmaf(-s, rkj, c * xj);
            }
        }
    }
    __device__ __forceinline__ float sqrt_det() const
    {
        float m = 1.f;
#pragma unroll
        for (int k = 0; k < 6; ++k) m *= r[at(k, k)];
        return fabsf(m);
    }
};

// ---------------------------------------------------------------- samplers (Sec. 4.3)
// Smoothing of particle n's noise: 0 raw samples, 1 cubic B-spline, 2 comb filter.
__device__ __forceinline__ int smoothing_of(const Problem& pb, int n)
{
    if (pb.filter == STORM_FILTER_COMB) return 2;
    if (pb.filter == STORM_FILTER_MIXED) return (n >= pb.n_null && n < pb.n_null + pb.n_bs) ? 1 : 2;
    return pb.nk > 0 ? 1 : 0;
}

// Comb filter of one (particle, joint) noise column in place, e[h * stride],
// h = 0..H-1: y_h = c0 e_h + c1 y_{h-1} + c2 y_{h-2}, zero before h = 0.
__device__ __forceinline__ void comb_column(float* e, int H, int stride, const float (&c)[3])
{
    float y1 = 0.f, y2 = 0.f;
    for (int h = 0; h < H; ++h) {
        const float y = fmaf(c[0], e[h * stride], fmaf(c[1], y1, c[2] * y2));
        e[h * stride] = y;
        y2 = y1;
        y1 = y;
    }
}

// ---------------------------------------------------------------- Eq. 8 twist
__device__ __forceinline__ void cross3(const float* a, const float* b, float* c)
{
    c[0] = fmaf(a[1], b[2], -a[2] * b[1]);
    c[1] = fmaf(a[2], b[0], -a[0] * b[2]);
    c[2] = fmaf(a[0], b[1], -a[1] * b[0]);
}

// End-effector velocity and acceleration, [linear; angular] at the end-effector
// point p, from the joint axes z[c] and origins o[c] (world frame):
// X_dot = sum_c theta_dot_c [z_c x (p - o_c); z_c] and X_ddot = J_dot theta_dot +
// J theta_ddot.  Joint by joint, w is the angular velocity of the link before
// joint c and v_o the velocity of o_c (v_o += w x (o_c - o_{c-1})); then
// z_c_dot = w x z_c and column c of J_dot is [z_c_dot x (p - o_c) + z_c x
// (p_dot - v_o); z_c_dot].
__device__ __forceinline__ void ee_twist(const float (&z)[kMaxDof][3], const float (&o)[kMaxDof][3],
                                         const float (&p)[3], const float* thd, const float* thdd, int d,
                                         float (&xd)[6], float (&xdd)[6])
{
    float zr[kMaxDof][3];
#pragma unroll
    for (int k = 0; k < 6; ++k) xd[k] = xdd[k] = 0.f;
#pragma unroll
    for (int c = 0; c < kMaxDof; ++c) {
        if (c < d) {
            const float r[3] = {p[0] - o[c][0], p[1] - o[c][1], p[2] - o[c][2]};
            cross3(z[c], r, zr[c]);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                xd[a] = fmaf(thd[c], zr[c][a], xd[a]);
                xd[3 + a] = fmaf(thd[c], z[c][a], xd[3 + a]);
            }
        }
    }
    float w[3] = {0.f, 0.f, 0.f}, vo[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < kMaxDof; ++c) {
        if (c < d) {
            if (c > 0) {
                const float dd[3] = {o[c][0] - o[c - 1][0], o[c][1] - o[c - 1][1], o[c][2] - o[c - 1][2]};
                float t[3];
                cross3(w, dd, t);
#pragma unroll
                for (int a = 0; a < 3; ++a) vo[a] += t[a];
            }
            float zd[3], t1[3], t2[3];
            cross3(w, z[c], zd);
            const float r[3] = {p[0] - o[c][0], p[1] - o[c][1], p[2] - o[c][2]};
            const float q[3] = {xd[0] - vo[0], xd[1] - vo[1], xd[2] - vo[2]};
            cross3(zd, r, t1);
            cross3(z[c], q, t2);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                xdd[a] = fmaf(thd[c], t1[a] + t2[a], fmaf(thdd[c], zr[c][a], xdd[a]));
                xdd[3 + a] = fmaf(thd[c], zd[a], fmaf(thdd[c], z[c][a], xdd[3 + a]));
                w[a] = fmaf(thd[c], z[c][a], w[a]);
            }
        }
    }
}

// The two task-space limit terms: max(0, |v| - v_max), max(0, |a| - a_max).
__device__ __forceinline__ float2 ee_limit_terms(const Problem& pb, const float (&xd)[6], const float (&xdd)[6])
{
    const float sp = sqrtf(fmaf(xd[0], xd[0], fmaf(xd[1], xd[1], xd[2] * xd[2])));
    const float ac = sqrtf(fmaf(xdd[0], xdd[0], fmaf(xdd[1], xdd[1], xdd[2] * xdd[2])));
    return make_float2(fmaxf(0.f, sp - pb.ee_vel_max), fmaxf(0.f, ac - pb.ee_acc_max));
}

// ---------------------------------------------------------------- ball on a tray
// The ball's in-plane state in the end-effector frame at the current robot
// state theta: x0 = R^T (b - p), v0 = R^T v_b -> (x0.x, x0.y, v0.x, v0.y).
__device__ __forceinline__ float4 ball_initial(const float* dhx, int d, const float* theta, const float* ball)
{
    float R[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
    float p[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < kMaxDof; ++i)
        if (i < d) dh_step(R, p, dhx[i * 8], dhx[i * 8 + 1], dhx[i * 8 + 2], dhx[i * 8 + 3], theta[i] + dhx[i * 8 + 4]);
    const float e[3] = {ball[0] - p[0], ball[1] - p[1], ball[2] - p[2]};
    return make_float4(fmaf(R[0], e[0], fmaf(R[3], e[1], R[6] * e[2])),
                       fmaf(R[1], e[0], fmaf(R[4], e[1], R[7] * e[2])),
                       fmaf(R[0], ball[3], fmaf(R[3], ball[4], R[6] * ball[5])),
                       fmaf(R[1], ball[3], fmaf(R[4], ball[4], R[7] * ball[5])));
}

// In-plane gravity in the end-effector frame of rotation R (row-major): (R^T g).xy.
__device__ __forceinline__ float2 ball_accel(const float (&R)[9], const float (&g)[3])
{
    return make_float2(fmaf(R[0], g[0], fmaf(R[3], g[1], R[6] * g[2])),
                       fmaf(R[1], g[0], fmaf(R[4], g[1], R[7] * g[2])));
}

// One particle's ball along the horizon (Eq. 7's semi-implicit recurrence on the
// in-plane accelerations a[h * 2 .. +1]); c[h] += w_ball * |x_h - tray|, and the
// unweighted term to term[h * term_stride] when term is not null.
__device__ __forceinline__ void ball_scan(int H, float w_ball, float tray_x, float tray_y, float4 s0, const float* a,
                                          const float* dt, float* c, float* term, int term_stride)
{
    float vx = s0.z, vy = s0.w, x = s0.x, y = s0.y;
    for (int h = 0; h < H; ++h) {
        vx = fmaf(dt[h], a[2 * h], vx);
        vy = fmaf(dt[h], a[2 * h + 1], vy);
        x = fmaf(dt[h], vx, x);
        y = fmaf(dt[h], vy, y);
        const float ex = x - tray_x, ey = y - tray_y;
        const float cb = sqrtf(fmaf(ex, ex, ey * ey));
        c[h] = fmaf(w_ball, cb, c[h]);
        if (term) term[static_cast<size_t>(h) * term_stride] = cb;
    }
}

__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.f), 1.f); }

// Squared distance between segments p0 + s (p1 - p0) and q0 + t (q1 - q0),
// s, t in [0, 1]: the stationary point of the squared distance for s, t
// inside, else the best t for the clamped s, or the best s at a clamped end of
// t.  Each clamp keeps one point the nearest to the other, so in the nearly
// parallel case, where the solve for s loses its digits, the result is off by
// at most the segment length times the sine of their angle (that angle being
// what makes the solve poor); the capsule radii are padded for it.
__device__ __forceinline__ float seg_seg_dist2(float3 p0, float3 p1, float3 q0, float3 q1)
{
    const float3 d1 = make_float3(p1.x - p0.x, p1.y - p0.y, p1.z - p0.z);
    const float3 d2 = make_float3(q1.x - q0.x, q1.y - q0.y, q1.z - q0.z);
    const float3 r = make_float3(p0.x - q0.x, p0.y - q0.y, p0.z - q0.z);
    const float a = fmaf(d1.x, d1.x, fmaf(d1.y, d1.y, d1.z * d1.z));
    const float e = fmaf(d2.x, d2.x, fmaf(d2.y, d2.y, d2.z * d2.z));
    const float b = fmaf(d1.x, d2.x, fmaf(d1.y, d2.y, d1.z * d2.z));
    const float c = fmaf(d1.x, r.x, fmaf(d1.y, r.y, d1.z * r.z));
    const float f = fmaf(d2.x, r.x, fmaf(d2.y, r.y, d2.z * r.z));
    float s = 0.f, t = 0.f;
    if (a > 1e-12f && e > 1e-12f) {
        const float den = fmaf(a, e, -b * b);
        s = den > 0.f ? clamp01(__fdividef(fmaf(b, f, -c * e), den)) : 0.f;
        t = __fdividef(fmaf(b, s, f), e);
        if (t < 0.f) {
            t = 0.f;
            s = clamp01(__fdividef(-c, a));
        } else if (t > 1.f) {
            t = 1.f;
            s = clamp01(__fdividef(b - c, a));
        }
    } else if (e > 1e-12f) {
        t = clamp01(__fdividef(f, e));
    } else if (a > 1e-12f) {
        s = clamp01(__fdividef(-c, a));
    }
    const float x = fmaf(d1.x, s, fmaf(-d2.x, t, r.x)), y = fmaf(d1.y, s, fmaf(-d2.y, t, r.y)),
                z = fmaf(d1.z, s, fmaf(-d2.z, t, r.z));
    return fmaf(x, x, fmaf(y, y, z * z));
}

}  // namespace storm
