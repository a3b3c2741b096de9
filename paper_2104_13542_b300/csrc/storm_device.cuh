// storm_device.cuh -- device-side building blocks of the STORM control step.
//
// Counter-based noise (Philox4x32-10 + Box-Muller), the modified-DH chain
// step, the manipulability score and the per-problem parameter block that
// every kernel receives by value.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace storm {

constexpr int kMaxDof = 7;
constexpr int kThreads = 256;        // default rollout CTA size
constexpr int kMaxThreads = 512;     // largest rollout CTA size the tuner may pick
constexpr int kUpdateThreads = 256;  // distribution-update CTA size (one CTA per horizon step)
constexpr int kLinkPairs = (kMaxDof + 1) * kMaxDof / 2;  // frame pairs (la < lb) of a chain

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
    int broadphase;          // 1: exact sphere tests only where the link bounds overlap
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
    const float* self_pred;  // N x H surrogate self distances (nullable)
    float self_margin;       // exact self check only where self_pred < self_margin
    // pair blocks of frames (la, lb), la < lb, are [lp_begin[t], lp_begin[t + 1]) with
    // t = link_pair_index(la, lb); the blocks are sorted by (la, lb)
    uint16_t lp_begin[kLinkPairs + 1];
};

// Step bookkeeping kept on the device so captured graphs need no host update.
struct StepState {
    uint32_t step;   // index of the next control step
    int status;      // OR of warnings of the current step
    float best;      // min total cost of the last iteration
    float wmean;     // weighted mean total cost of the last iteration
};

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
__device__ __forceinline__ void dh_step(float (&R)[9], float (&p)[3], float a, float ca, float sa,
                                        float dd, float theta)
{
    float st, ct;
    sincosf(theta, &st, &ct);
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

}  // namespace storm
