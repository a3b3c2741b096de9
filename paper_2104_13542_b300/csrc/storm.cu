// storm.cu -- kernels, host runtime and C ABI of the B300 STORM control step.
//
// Hot path of one control step (Algorithm 1 of the paper):
//   k_shift                      shift of the mean (skipped at step 0)
//   K x { k_rollout, k_update }  sample_controls + generate_rollouts, update_distribution
// The sequence is captured once into a CUDA graph per handle and replayed each
// step; host<->device traffic per step is one 4*(3d+7)-byte copy in and one
// 4*d + 16-byte copy out.
#include "storm.h"
#include "storm_device.cuh"

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <utility>
#include <mutex>
#include <set>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

using namespace storm;

// ============================================================================ layout

struct RolloutLayout {
    int tab, frame, boxlh;                                  // 16-byte arrays
    int mu, sigma, eps, u, th, thd, part, dself, dworld, goal, state, ba, ball0;  // float arrays
    int slink;                                              // int arrays
    int bytes;
};

__host__ __device__ inline int take_(int& off, int bytes)
{
    const int o = off;
    off += (bytes + 15) & ~15;
    return o;
}

// Shared-memory plan of one rollout CTA (identical on host and device): a copy
// of the per-problem tables, then the CTA's working arrays.
__host__ __device__ inline RolloutLayout rollout_layout(const Problem& pb)
{
    RolloutLayout L;
    int off = 0;
    const int I = pb.ppc * pb.H;
    L.tab = take_(off, pb.table_bytes);
    L.frame = take_(off, I * (pb.d + 1) * 3 * 16);
    L.boxlh = take_(off, pb.B * 2 * 16);
    L.mu = take_(off, pb.H * pb.d * 4);
    L.sigma = take_(off, pb.d * 4);
    L.eps = take_(off, pb.ppc * pb.S * pb.d * 4);
    L.u = take_(off, pb.ppc * pb.H * pb.d * 4);
    L.th = take_(off, pb.ppc * pb.H * pb.d * 4);
    L.thd = take_(off, pb.ppc * pb.H * pb.d * 4);
    L.part = take_(off, I * 4);
    L.dself = take_(off, I * 4);
    L.dworld = take_(off, I * 4);
    L.goal = take_(off, 12 * 4);
    L.state = take_(off, 3 * pb.d * 4);
    L.ba = take_(off, I * 2 * 4);   // ball: in-plane gravity per item
    L.ball0 = take_(off, 4 * 4);    // ball: initial in-plane state
    L.slink = take_(off, pb.M * 4);
    L.bytes = off;
    return L;
}

// Where table `p` of the device table block lands in the shared-memory copy.
template <typename T>
__device__ __forceinline__ const T* in_copy(const unsigned char* copy, const uint4* base, const T* p)
{
    return reinterpret_cast<const T*>(copy + (reinterpret_cast<const unsigned char*>(p) -
                                              reinterpret_cast<const unsigned char*>(base)));
}

struct RolloutOut {
    float* u;          // N x H x d (required)
    float* theta;      // optional N x H x d
    float* theta_dot;  // optional N x H x d
    float* ee;         // optional N x H x 12
    float* terms;      // optional N x H x 8
    float* cost;       // optional N x H
    float* Ctot;       // N (required)
};

// ============================================================================ kernels

// sample_controls + generate_rollouts of particles [n0, n0 + np) in one CTA.
// Phases: stage tables -> noise -> smoothed controls -> per-(particle, joint)
// integration scan (Eq. 7) -> per-(particle, step) FK, Jacobian and
// non-collision cost terms (Eqs. 8-12), link frames to shared memory ->
// per-(step, sphere) sphere centre and world collision (Eq. 14 reading) ->
// per-(pair, step) self collision (Eq. 13 reading) -> running cost (Eq. 15)
// and discounted totals (Eq. 2).
__device__ __forceinline__ void rollout_particles(const Problem& pb, const RolloutOut& out,
                                                  const float* __restrict__ state,
                                                  const float* __restrict__ goal, uint32_t step,
                                                  int iter, int n0, int np, unsigned char* smem)
{
    const RolloutLayout L = rollout_layout(pb);
    float4* s_frame = reinterpret_cast<float4*>(smem + L.frame);
    float4* s_boxlh = reinterpret_cast<float4*>(smem + L.boxlh);
    float* s_mu = reinterpret_cast<float*>(smem + L.mu);
    float* s_sigma = reinterpret_cast<float*>(smem + L.sigma);
    float* s_eps = reinterpret_cast<float*>(smem + L.eps);
    float* s_u = reinterpret_cast<float*>(smem + L.u);
    float* s_th = reinterpret_cast<float*>(smem + L.th);
    float* s_thd = reinterpret_cast<float*>(smem + L.thd);
    float* s_part = reinterpret_cast<float*>(smem + L.part);
    float* s_dself = reinterpret_cast<float*>(smem + L.dself);
    float* s_dworld = reinterpret_cast<float*>(smem + L.dworld);
    float* s_goal = reinterpret_cast<float*>(smem + L.goal);
    float* s_state = reinterpret_cast<float*>(smem + L.state);
    int* s_slink = reinterpret_cast<int*>(smem + L.slink);

    const int tid = threadIdx.x, nt = blockDim.x;
    const int d = pb.d, H = pb.H, S = pb.S, M = pb.M, F = pb.d + 1;
    const int I = np * H;
    const int HD = H * d;
    trace_stamp(pb.trace, 0);

    // ---- stage: the per-problem tables in one vectorised copy, then mu, sigma,
    // the state and the goal rotation
    {
        const uint4* src = pb.tables;
        uint4* dst = reinterpret_cast<uint4*>(smem + L.tab);
        for (int i = tid; i < pb.table_bytes / 16; i += nt) dst[i] = src[i];
    }
    const int mu_off = (pb.shift_view && step > 0) ? d : 0;  // the shifted mean at a step's start
    for (int i = tid; i < HD; i += nt) s_mu[i] = i + mu_off < HD ? __ldcg(pb.mu + i + mu_off) : 0.f;
    for (int i = tid; i < d; i += nt) s_sigma[i] = __ldcg(pb.sigma + i);
    for (int i = tid; i < 3 * d; i += nt) s_state[i] = state[i];
    if (tid == 0) {
        // goal rotation R_g (row-major) from the normalised quaternion, then p_g
        const float qn = rsqrtf(goal[3] * goal[3] + goal[4] * goal[4] + goal[5] * goal[5] +
                                goal[6] * goal[6]);
        const float w = goal[3] * qn, x = goal[4] * qn, y = goal[5] * qn, z = goal[6] * qn;
        s_goal[0] = 1.f - 2.f * (y * y + z * z);
        s_goal[1] = 2.f * (x * y - w * z);
        s_goal[2] = 2.f * (x * z + w * y);
        s_goal[3] = 2.f * (x * y + w * z);
        s_goal[4] = 1.f - 2.f * (x * x + z * z);
        s_goal[5] = 2.f * (y * z - w * x);
        s_goal[6] = 2.f * (x * z - w * y);
        s_goal[7] = 2.f * (y * z + w * x);
        s_goal[8] = 1.f - 2.f * (x * x + y * y);
        s_goal[9] = goal[0];
        s_goal[10] = goal[1];
        s_goal[11] = goal[2];
    }
    __syncthreads();
    const unsigned char* tab = smem + L.tab;
    const float* s_dhx = in_copy(tab, pb.tables, pb.dhx);
    const float* s_qlo = in_copy(tab, pb.tables, pb.qlo);
    const float* s_qhi = in_copy(tab, pb.tables, pb.qhi);
    const float4* s_sph = in_copy(tab, pb.tables, pb.sph);
    const int* s_first = in_copy(tab, pb.tables, pb.link_first);
    const uint32_t* s_pairs = in_copy(tab, pb.tables, pb.pairs);
    const uint4* s_pblk = in_copy(tab, pb.tables, pb.pblk);
    const float4* s_lb = in_copy(tab, pb.tables, pb.lbound);
    const float* s_boxes = in_copy(tab, pb.tables, pb.boxes);
    const float4* s_wsph = in_copy(tab, pb.tables, pb.wsph);
    const float* s_dt = in_copy(tab, pb.tables, pb.dt);
    const float* s_gpow = in_copy(tab, pb.tables, pb.gpow);
    const float* s_vmax = in_copy(tab, pb.tables, pb.vmax);
    const float* s_basis = in_copy(tab, pb.tables, pb.basis);
    // derived per-CTA tables (read after the next barrier)
    for (int i = tid; i < M; i += nt) {
        int f = 0;
        while (f < d && i >= s_first[f + 1]) ++f;
        s_slink[i] = f;
    }
    for (int i = tid; i < pb.B; i += nt) {
        const float* b = s_boxes + i * 6;
        s_boxlh[2 * i] = make_float4(b[0] - b[3], b[1] - b[4], b[2] - b[5], 0.f);
        s_boxlh[2 * i + 1] = make_float4(b[0] + b[3], b[1] + b[4], b[2] + b[5], 0.f);
    }

    // ---- noise eps[n][s][j] for this CTA's particles
    const int per = S * d;
    if (pb.sampler == STORM_SAMPLER_PHILOX) {
        const uint32_t e0 = static_cast<uint32_t>(n0) * per;
        const uint32_t e1 = static_cast<uint32_t>(n0 + np) * per;
        const uint32_t b0 = e0 >> 2, b1 = (e1 + 3) >> 2;
        const uint32_t c2 = (pb.instance << 8) | static_cast<uint32_t>(iter);
        for (uint32_t b = b0 + tid; b < b1; b += nt) {
            const uint4 x = philox4x32_10(make_uint4(b, step, c2, 0u), pb.seed_lo, pb.seed_hi);
            const float2 z01 = gauss_pair(x.x, x.y);
            const float2 z23 = gauss_pair(x.z, x.w);
            const float z[4] = {z01.x, z01.y, z23.x, z23.y};
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const uint32_t e = 4 * b + l;
                if (e >= e0 && e < e1) s_eps[e - e0] = z[l];
            }
        }
    } else {
        for (int i = tid; i < np * per; i += nt) s_eps[i] = pb.halton[static_cast<size_t>(n0) * per + i];
    }
    __syncthreads();
    if (pb.filter != STORM_FILTER_DEFAULT) {  // comb-filtered particles, one sample per step (S = H)
        for (int t = tid; t < np * d; t += nt) {
            const int p = t / d, j = t - p * d;
            if (smoothing_of(pb, n0 + p) == 2) comb_column(s_eps + p * S * d + j, H, d, pb.comb);
        }
        __syncthreads();
    }
    trace_stamp(pb.trace, 1);

    // ---- controls u = mu + sigma o (B eps), null particles zero
    for (int i = tid; i < np * HD; i += nt) {
        const int p = i / HD, r = i - p * HD, h = r / d, j = r - h * d;
        float e;
        if (smoothing_of(pb, n0 + p) == 1) {
            e = 0.f;
            for (int s = 0; s < pb.nk; ++s) e = fmaf(s_basis[h * pb.nk + s], s_eps[(p * S + s) * d + j], e);
        } else {
            e = s_eps[(p * S + h) * d + j];
        }
        const float uu = (n0 + p < pb.n_null) ? 0.f : fmaf(s_sigma[j], e, s_mu[h * d + j]);
        s_u[i] = uu;
        out.u[static_cast<size_t>(n0) * HD + i] = uu;
    }
    __syncthreads();

    // ---- integration scan per (particle, joint), Eq. 7
    for (int t = tid; t < np * d; t += nt) {
        const int p = t / d, j = t - p * d;
        float v = s_state[d + j], q = s_state[j];
        for (int h = 0; h < H; ++h) {
            const int idx = (p * H + h) * d + j;
            v = fmaf(s_dt[h], s_u[idx], v);
            q = fmaf(s_dt[h], v, q);
            s_thd[idx] = v;
            s_th[idx] = q;
        }
    }
    __syncthreads();
    trace_stamp(pb.trace, 2);
    if (out.theta)
        for (int i = tid; i < np * HD; i += nt) out.theta[static_cast<size_t>(n0) * HD + i] = s_th[i];
    if (out.theta_dot)
        for (int i = tid; i < np * HD; i += nt)
            out.theta_dot[static_cast<size_t>(n0) * HD + i] = s_thd[i];

    // ---- per (particle, step): FK frames, Jacobian, non-collision costs
    const bool want_ee = pb.w_ee_vel != 0.f || pb.w_ee_acc != 0.f || out.terms;
    const bool ball_on = pb.ball && pb.w_ball != 0.f;
    float* s_ba = reinterpret_cast<float*>(smem + L.ba);
    float4* s_ball0 = reinterpret_cast<float4*>(smem + L.ball0);
    if (ball_on && tid == 0) *s_ball0 = ball_initial(s_dhx, d, s_state, pb.ball);
    for (int item = tid; item < I; item += nt) {
        const int p = item / H, h = item - p * H;
        const float* th = s_th + (p * H + h) * d;
        const float* thd = s_thd + (p * H + h) * d;
        const float* uh = s_u + (p * H + h) * d;
        const float* up = (h == 0) ? s_state + 2 * d : uh - d;
        float4* fr = s_frame + item * F * 3;

        float R[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
        float pp[3] = {0.f, 0.f, 0.f};
        fr[0] = make_float4(1.f, 0.f, 0.f, 0.f);
        fr[1] = make_float4(0.f, 1.f, 0.f, 0.f);
        fr[2] = make_float4(0.f, 0.f, 1.f, 0.f);
#pragma unroll
        for (int i = 0; i < kMaxDof; ++i) {
            if (i < d) {
                const float* dh = s_dhx + i * 8;
                dh_step(R, pp, dh[0], dh[1], dh[2], dh[3], th[i] + dh[4]);
#pragma unroll
                for (int r = 0; r < 3; ++r)
                    fr[(i + 1) * 3 + r] = make_float4(R[r * 3 + 0], R[r * 3 + 1], R[r * 3 + 2], pp[r]);
            }
        }

        // pose (Eq. 9): position in the goal frame, weighted per axis
        const float dx = pp[0] - s_goal[9], dy = pp[1] - s_goal[10], dz = pp[2] - s_goal[11];
        float c_pos = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float e = pb.pos_w[a] * fmaf(s_goal[a], dx, fmaf(s_goal[3 + a], dy, s_goal[6 + a] * dz));
            c_pos = fmaf(e, e, c_pos);
        }
        c_pos = sqrtf(c_pos);
        float c_rot = 0.f;
        if (pb.rot_mode == STORM_ROT_QUAT) {
            // |q_ee . q_g| = sqrt(1 + tr(R_g^T R_ee)) / 2
            float tr = 0.f;
#pragma unroll
            for (int k = 0; k < 9; ++k) tr = fmaf(s_goal[k], R[k], tr);
            c_rot = 1.f - 0.5f * sqrtf(fmaxf(0.f, 1.f + tr));
        } else {
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float rtr =
                        fmaf(s_goal[r], R[c], fmaf(s_goal[3 + r], R[3 + c], s_goal[6 + r] * R[6 + c]));
                    const float e = ((r == c) ? 1.f : 0.f) - rtr;
                    const float we = e * pb.rot_w[c];
                    c_rot = fmaf(we, we, c_rot);
                }
            c_rot = sqrtf(c_rot);
        }
        // stop (Eq. 10), joint limits (Eq. 11), smoothness
        float c_stop = 0.f, c_joint = 0.f, c_smooth = 0.f;
        const float vlim = s_vmax[h];
        for (int j = 0; j < d; ++j) {
            const float vs = fmaxf(0.f, fabsf(thd[j]) - vlim);
            c_stop = fmaf(vs, vs, c_stop);
            const float vj = fmaxf(0.f, s_qlo[j] - th[j]) + fmaxf(0.f, th[j] - s_qhi[j]);
            c_joint = fmaf(vj, vj, c_joint);
            const float du = uh[j] - up[j];
            c_smooth = fmaf(du, du, c_smooth);
        }
        c_stop = sqrtf(c_stop);
        c_joint = sqrtf(c_joint);
        // (manipulability, Eq. 12, is added in the collision phase)
        float part = pb.w_pos * c_pos + pb.w_rot * c_rot + pb.w_stop * c_stop + pb.w_joint * c_joint +
                     pb.w_smooth * c_smooth;
        float2 c_ee = make_float2(0.f, 0.f);
        if (want_ee) {  // task-space limits on X_dot, X_ddot (Eq. 8), theta_ddot = u
            float zc[kMaxDof][3], oc[kMaxDof][3];  // joint axes and origins, from the frames
#pragma unroll
            for (int i = 0; i < kMaxDof; ++i) {
                if (i < d) {
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        const float4 row = fr[(i + 1) * 3 + r];
                        zc[i][r] = row.z;
                        oc[i][r] = row.w;
                    }
                } else {
                    zc[i][0] = zc[i][1] = zc[i][2] = oc[i][0] = oc[i][1] = oc[i][2] = 0.f;
                }
            }
            float xd[6], xdd[6];
            ee_twist(zc, oc, pp, thd, uh, d, xd, xdd);
            c_ee = ee_limit_terms(pb, xd, xdd);
            if (pb.w_ee_vel != 0.f) part = fmaf(pb.w_ee_vel, c_ee.x, part);
            if (pb.w_ee_acc != 0.f) part = fmaf(pb.w_ee_acc, c_ee.y, part);
        }
        if (ball_on) {
            const float2 a = ball_accel(R, pb.grav);
            s_ba[2 * item] = a.x;
            s_ba[2 * item + 1] = a.y;
        }
        s_part[item] = part;
        s_dself[item] = 0.f;
        s_dworld[item] = 0.f;
        const size_t g = static_cast<size_t>(n0) * H + item;
        if (out.ee) {
            float* e = out.ee + g * 12;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                e[r * 4 + 0] = R[r * 3 + 0];
                e[r * 4 + 1] = R[r * 3 + 1];
                e[r * 4 + 2] = R[r * 3 + 2];
                e[r * 4 + 3] = pp[r];
            }
        }
        if (out.terms) {
            float* t = out.terms + g * STORM_NTERMS;
            t[0] = c_pos;
            t[1] = c_rot;
            t[2] = c_stop;
            t[3] = c_joint;
            t[7] = c_smooth;
            t[8] = c_ee.x;
            t[9] = c_ee.y;
            t[10] = 0.f;
        }
    }
    __syncthreads();
    trace_stamp(pb.trace, 3);

    // ---- world collision, Eq. 14 reading.  Broad phase: per (step, link) the
    // link's bounding sphere against every obstacle, and the exact per-sphere
    // test (below) only for the obstacles it touches.  Brute force otherwise:
    // per (step, sphere) against every obstacle.  Both give the same depths.
    // Manipulability (Eq. 12) shares this phase: its long dependent chain is
    // hidden behind the other warps' collision work.  The geometric Jacobian
    // is taken about the base origin, columns [o_i x z_i; z_i] -- det(J J^T)
    // does not depend on the reference point (J(p) = [[I, -[p]x], [0, I]] J(0)).
    const bool want_manip = pb.w_manip != 0.f || out.terms;
    const int NMU = want_manip ? I : 0;
    // one manipulability unit per thread, taken by the last threads of the CTA
    for (int item = nt - 1 - tid; item < NMU && item >= 0; item += nt) {
        const float4* fr = s_frame + item * F * 3;
        float J[6][kMaxDof];
#pragma unroll
        for (int i = 0; i < kMaxDof; ++i) {
            if (i < d) {
                const float4 r0 = fr[(i + 1) * 3], r1 = fr[(i + 1) * 3 + 1], r2 = fr[(i + 1) * 3 + 2];
                J[0][i] = r1.w * r2.z - r2.w * r1.z;
                J[1][i] = r2.w * r0.z - r0.w * r2.z;
                J[2][i] = r0.w * r1.z - r1.w * r0.z;
                J[3][i] = r0.z;
                J[4][i] = r1.z;
                J[5][i] = r2.z;
            } else {
#pragma unroll
                for (int r = 0; r < 6; ++r) J[r][i] = 0.f;
            }
        }
        const float m = manipulability_mgs(J, d);
        const float c_manip = (m < pb.k_m) ? 1.f - m : 0.f;
        s_part[item] += pb.w_manip * c_manip;  // this unit alone writes s_part here
        if (out.terms) out.terms[(static_cast<size_t>(n0) * H + item) * STORM_NTERMS + 4] = c_manip;
    }
    if (pb.broadphase) {
        for (int idx = tid; idx < I * F; idx += nt) {
            const int item = idx / F, f = idx - item * F;
            const int s0 = s_first[f], s1 = s_first[f + 1];
            if (s0 == s1) continue;
            const float4* T = s_frame + (item * F + f) * 3;
            const float4 r0 = T[0], r1 = T[1], r2 = T[2];
            const float4 lb = s_lb[f];
            const float bx = fmaf(r0.x, lb.x, fmaf(r0.y, lb.y, fmaf(r0.z, lb.z, r0.w)));
            const float by = fmaf(r1.x, lb.x, fmaf(r1.y, lb.y, fmaf(r1.z, lb.z, r1.w)));
            const float bz = fmaf(r2.x, lb.x, fmaf(r2.y, lb.y, fmaf(r2.z, lb.z, r2.w)));
            const float R2 = lb.w * lb.w;
            float depth = 0.f;
            for (int b = 0; b < pb.B; ++b) {
                const float4 lo = s_boxlh[2 * b], hi = s_boxlh[2 * b + 1];
                const float ex = bx - fminf(fmaxf(bx, lo.x), hi.x);
                const float ey = by - fminf(fmaxf(by, lo.y), hi.y);
                const float ez = bz - fminf(fmaxf(bz, lo.z), hi.z);
                if (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) >= R2) continue;
                const float* box = s_boxes + b * 6;
                for (int s = s0; s < s1; ++s) {
                    const float4 q = s_sph[s];
                    const float cx = fmaf(r0.x, q.x, fmaf(r0.y, q.y, fmaf(r0.z, q.z, r0.w)));
                    const float cy = fmaf(r1.x, q.x, fmaf(r1.y, q.y, fmaf(r1.z, q.z, r1.w)));
                    const float cz = fmaf(r2.x, q.x, fmaf(r2.y, q.y, fmaf(r2.z, q.z, r2.w)));
                    const float fx = cx - fminf(fmaxf(cx, lo.x), hi.x);
                    const float fy = cy - fminf(fmaxf(cy, lo.y), hi.y);
                    const float fz = cz - fminf(fmaxf(cz, lo.z), hi.z);
                    if (fmaf(fx, fx, fmaf(fy, fy, fz * fz)) < q.w * q.w) {
                        const float qx = fabsf(cx - box[0]) - box[3];
                        const float qy = fabsf(cy - box[1]) - box[4];
                        const float qz = fabsf(cz - box[2]) - box[5];
                        const float ox = fmaxf(qx, 0.f), oy = fmaxf(qy, 0.f), oz = fmaxf(qz, 0.f);
                        const float sd = sqrtf(fmaf(ox, ox, fmaf(oy, oy, oz * oz))) +
                                         fminf(fmaxf(qx, fmaxf(qy, qz)), 0.f) - q.w;
                        depth = fmaxf(depth, -sd);
                    }
                }
            }
            for (int k = 0; k < pb.O; ++k) {
                const float4 w = s_wsph[k];
                const float ex = bx - w.x, ey = by - w.y, ez = bz - w.z;
                const float rb = lb.w + w.w;
                if (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) >= rb * rb) continue;
                for (int s = s0; s < s1; ++s) {
                    const float4 q = s_sph[s];
                    const float cx = fmaf(r0.x, q.x, fmaf(r0.y, q.y, fmaf(r0.z, q.z, r0.w)));
                    const float cy = fmaf(r1.x, q.x, fmaf(r1.y, q.y, fmaf(r1.z, q.z, r1.w)));
                    const float cz = fmaf(r2.x, q.x, fmaf(r2.y, q.y, fmaf(r2.z, q.z, r2.w)));
                    const float gx = cx - w.x, gy = cy - w.y, gz = cz - w.z;
                    const float dist2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
                    const float rs = q.w + w.w;
                    if (dist2 < rs * rs) depth = fmaxf(depth, rs - sqrtf(dist2));
                }
            }
            if (depth > 0.f) atomicMax(reinterpret_cast<int*>(s_dworld + item), __float_as_int(depth));
        }
    } else
    for (int idx = tid; idx < I * M; idx += nt) {
        const int item = idx / M, s = idx - item * M;
        const float4 q = s_sph[s];
        const float4* T = s_frame + (item * F + s_slink[s]) * 3;
        const float4 r0 = T[0], r1 = T[1], r2 = T[2];
        float4 c;
        c.x = fmaf(r0.x, q.x, fmaf(r0.y, q.y, fmaf(r0.z, q.z, r0.w)));
        c.y = fmaf(r1.x, q.x, fmaf(r1.y, q.y, fmaf(r1.z, q.z, r1.w)));
        c.z = fmaf(r2.x, q.x, fmaf(r2.y, q.y, fmaf(r2.z, q.z, r2.w)));
        c.w = q.w;
        const float r2s = c.w * c.w;
        float depth = 0.f;
        for (int b = 0; b < pb.B; ++b) {
            const float4 lo = s_boxlh[2 * b], hi = s_boxlh[2 * b + 1];
            const float ex = c.x - fminf(fmaxf(c.x, lo.x), hi.x);
            const float ey = c.y - fminf(fmaxf(c.y, lo.y), hi.y);
            const float ez = c.z - fminf(fmaxf(c.z, lo.z), hi.z);
            const float out2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
            if (out2 < r2s) {
                const float* bx = s_boxes + b * 6;
                const float qx = fabsf(c.x - bx[0]) - bx[3];
                const float qy = fabsf(c.y - bx[1]) - bx[4];
                const float qz = fabsf(c.z - bx[2]) - bx[5];
                const float ox = fmaxf(qx, 0.f), oy = fmaxf(qy, 0.f), oz = fmaxf(qz, 0.f);
                const float sd = sqrtf(fmaf(ox, ox, fmaf(oy, oy, oz * oz))) +
                                 fminf(fmaxf(qx, fmaxf(qy, qz)), 0.f) - c.w;
                depth = fmaxf(depth, -sd);
            }
        }
        for (int k = 0; k < pb.O; ++k) {
            const float4 w = s_wsph[k];
            const float ex = c.x - w.x, ey = c.y - w.y, ez = c.z - w.z;
            const float dist2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
            const float rs = c.w + w.w;
            if (dist2 < rs * rs) depth = fmaxf(depth, rs - sqrtf(dist2));
        }
        if (depth > 0.f) atomicMax(reinterpret_cast<int*>(s_dworld + item), __float_as_int(depth));
    }
    __syncthreads();
    trace_stamp(pb.trace, 4);
    // ---- self collision, Eq. 13 reading.  Pair blocks (every sphere of one
    // link against up to 8 spheres of another) keep the 8 centres in registers
    // while streaming the first link's spheres; leftover pairs one by one.  (A
    // problem with the learned self-collision network runs k_rollout_mlp.)
    for (int idx = tid; idx < I * pb.NPB; idx += nt) {
        const int item = idx / pb.NPB, bk = idx - item * pb.NPB;
        const uint4 blk = s_pblk[bk];  // a0, a1, b0, nb
        const int la = s_slink[blk.x], lbk = s_slink[blk.z];
        const float4* fa = s_frame + (item * F + la) * 3;
        const float4* fb = s_frame + (item * F + lbk) * 3;
        if (pb.broadphase) {  // the two links' bounding spheres apart: no sphere pair touches
            const float4 ba = s_lb[la], bb = s_lb[lbk];
            const float ex = (fmaf(fa[0].x, ba.x, fmaf(fa[0].y, ba.y, fmaf(fa[0].z, ba.z, fa[0].w)))) -
                             (fmaf(fb[0].x, bb.x, fmaf(fb[0].y, bb.y, fmaf(fb[0].z, bb.z, fb[0].w))));
            const float ey = (fmaf(fa[1].x, ba.x, fmaf(fa[1].y, ba.y, fmaf(fa[1].z, ba.z, fa[1].w)))) -
                             (fmaf(fb[1].x, bb.x, fmaf(fb[1].y, bb.y, fmaf(fb[1].z, bb.z, fb[1].w))));
            const float ez = (fmaf(fa[2].x, ba.x, fmaf(fa[2].y, ba.y, fmaf(fa[2].z, ba.z, fa[2].w)))) -
                             (fmaf(fb[2].x, bb.x, fmaf(fb[2].y, bb.y, fmaf(fb[2].z, bb.z, fb[2].w))));
            const float rr = ba.w + bb.w;
            if (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) >= rr * rr) continue;
        }
        float4 cb[8];
        {
            const float4 r0 = fb[0], r1 = fb[1], r2 = fb[2];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (k < static_cast<int>(blk.w)) {
                    const float4 q = s_sph[blk.z + k];
                    cb[k] = make_float4(fmaf(r0.x, q.x, fmaf(r0.y, q.y, fmaf(r0.z, q.z, r0.w))),
                                        fmaf(r1.x, q.x, fmaf(r1.y, q.y, fmaf(r1.z, q.z, r1.w))),
                                        fmaf(r2.x, q.x, fmaf(r2.y, q.y, fmaf(r2.z, q.z, r2.w))), q.w);
                } else {
                    cb[k] = make_float4(1e30f, 1e30f, 1e30f, 0.f);
                }
            }
        }
        const float4 r0 = fa[0], r1 = fa[1], r2 = fa[2];
        float depth = 0.f;
        for (uint32_t a = blk.x; a < blk.y; ++a) {
            const float4 q = s_sph[a];
            const float cx = fmaf(r0.x, q.x, fmaf(r0.y, q.y, fmaf(r0.z, q.z, r0.w)));
            const float cy = fmaf(r1.x, q.x, fmaf(r1.y, q.y, fmaf(r1.z, q.z, r1.w)));
            const float cz = fmaf(r2.x, q.x, fmaf(r2.y, q.y, fmaf(r2.z, q.z, r2.w)));
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float ex = cx - cb[k].x, ey = cy - cb[k].y, ez = cz - cb[k].z;
                const float dist2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                const float rs = q.w + cb[k].w;
                if (dist2 < rs * rs) depth = fmaxf(depth, rs - sqrtf(dist2));
            }
        }
        if (depth > 0.f) atomicMax(reinterpret_cast<int*>(s_dself + item), __float_as_int(depth));
    }
    for (int k = tid; k < pb.P; k += nt) {
        const uint32_t pr = s_pairs[k];
        const int a = pr & 0xffff, b = pr >> 16;
        const float4 qa = s_sph[a], qb = s_sph[b];
        const float rs = qa.w + qb.w;
        const float rs2 = rs * rs;
        for (int item = 0; item < I; ++item) {
            const float4* fa = s_frame + (item * F + s_slink[a]) * 3;
            const float4* fb = s_frame + (item * F + s_slink[b]) * 3;
            const float ex = (fmaf(fa[0].x, qa.x, fmaf(fa[0].y, qa.y, fmaf(fa[0].z, qa.z, fa[0].w)))) -
                             (fmaf(fb[0].x, qb.x, fmaf(fb[0].y, qb.y, fmaf(fb[0].z, qb.z, fb[0].w))));
            const float ey = (fmaf(fa[1].x, qa.x, fmaf(fa[1].y, qa.y, fmaf(fa[1].z, qa.z, fa[1].w)))) -
                             (fmaf(fb[1].x, qb.x, fmaf(fb[1].y, qb.y, fmaf(fb[1].z, qb.z, fb[1].w))));
            const float ez = (fmaf(fa[2].x, qa.x, fmaf(fa[2].y, qa.y, fmaf(fa[2].z, qa.z, fa[2].w)))) -
                             (fmaf(fb[2].x, qb.x, fmaf(fb[2].y, qb.y, fmaf(fb[2].z, qb.z, fb[2].w))));
            const float dist2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
            if (dist2 < rs2)
                atomicMax(reinterpret_cast<int*>(s_dself + item), __float_as_int(rs - sqrtf(dist2)));
        }
    }
    __syncthreads();

    trace_stamp(pb.trace, 5);
    // ---- running cost (Eq. 15)
    for (int item = tid; item < I; item += nt) {
        const float c = s_part[item] + pb.w_coll * (s_dself[item] + s_dworld[item]);
        s_part[item] = c;
        const size_t g = static_cast<size_t>(n0) * H + item;
        if (out.terms) {
            out.terms[g * STORM_NTERMS + 5] = s_dself[item];
            out.terms[g * STORM_NTERMS + 6] = s_dworld[item];
        }
    }
    __syncthreads();
    if (ball_on) {  // the ball along each particle's horizon
        for (int p = tid; p < np; p += nt)
            ball_scan(H, pb.w_ball, pb.tray[0], pb.tray[1], *s_ball0, s_ba + 2 * p * H, s_dt, s_part + p * H,
                      out.terms ? out.terms + (static_cast<size_t>(n0 + p) * H) * STORM_NTERMS + 10 : nullptr,
                      STORM_NTERMS);
        __syncthreads();
    }
    if (out.cost)
        for (int item = tid; item < I; item += nt) out.cost[static_cast<size_t>(n0) * H + item] = s_part[item];
    // ---- discounted total (Eq. 2)
    for (int p = tid; p < np; p += nt) {
        float C = 0.f;
        for (int h = 0; h < H; ++h) C = fmaf(s_gpow[h], s_part[p * H + h], C);
        out.Ctot[n0 + p] = C;
    }
    trace_stamp(pb.trace, 6);
}

__global__ void __launch_bounds__(kMaxThreads)
k_rollout(Problem pb, RolloutOut out, const float* __restrict__ state,
          const float* __restrict__ goal, const StepState* __restrict__ st, int step_override,
          int iter)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int n0 = blockIdx.x * pb.ppc;
    const int np = min(pb.ppc, pb.N - n0);
    pdl_trigger();
    pdl_wait();
    if (np <= 0) return;
    const uint32_t step = step_override >= 0 ? static_cast<uint32_t>(step_override) : st->step;
    rollout_particles(pb, out, state, goal, step, iter, n0, np, smem);
}

#include "storm_rollout_warp.cuh"

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum: fixed butterfly per warp, then warp 0 over warps.
__device__ float block_sum(float v, float* sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        float x = lane < nw ? sh[lane] : 0.f;
        x = warp_sum(x);
        if (lane == 0) sh[0] = x;
    }
    __syncthreads();
    return sh[0];
}

// Block-wide (min value, lowest index) over all threads; result in every thread.
__device__ void block_argmin(float& bv, int& bi, float* shf, int* shi)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov < bv || (ov == bv && oi < bi)) {
            bv = ov;
            bi = oi;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) {
        shf[wid] = bv;
        shi[wid] = bi;
    }
    __syncthreads();
    if (wid == 0) {
        bv = lane < nw ? shf[lane] : INFINITY;
        bi = lane < nw ? shi[lane] : INT_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov < bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            shf[0] = bv;
            shi[0] = bi;
        }
    }
    __syncthreads();
    bv = shf[0];
    bi = shi[0];
}

// update_distribution (Eqs. 4-6) on one thread-block cluster of kUpdCluster
// CTAs per problem, as weighted sums over the particles of the N x (H d)
// control matrix (one row per particle, contiguous).  The columns (h, j) are
// split into kUpdCluster contiguous ranges, one per CTA, so that all of a
// column's sums over the N particles are formed inside one CTA.  Every CTA
// finds the minimum cost of all N particles and forms all N weights (Eq. 6)
// and their sums -- the same operations in every CTA, so the same bits; its
// threads, one column and one of G interleaved particle groups each, sum
// w (u - mu_old), the groups added in order, into the new mean of its columns
// (Eq. 4), then, from the values still in registers, w (u - mu_new)^2 into each
// column's squared deviation, which the CTA adds per joint over its columns
// (Eq. 5).  One cluster barrier: ahead of it each CTA stores its per-joint
// sums (and, at the last iteration, the new mean's first row) into rank 0's
// shared memory; after it each CTA writes its columns of the mean (every CTA
// has read the old mean by then) and rank 0 forms sigma, records the
// iteration's best and weighted-mean cost and, at the last iteration of a
// step, writes next_command and advances the step counter.  Every sum runs in
// a fixed order: bitwise reproducible, whatever the grid around the cluster.
constexpr int kUpdCluster = 8;
constexpr int kUpdBatch = 32;     // loads in flight per thread
constexpr int kUpdCostRegs = 2;   // costs a thread loads ahead (N <= 1024 in one round)
constexpr int kUpdMaxCols = (STORM_MAX_H * kMaxDof + kUpdCluster - 1) / kUpdCluster;  // columns of one CTA
static_assert(kUpdMaxCols <= kUpdateThreads, "a thread per column of a CTA");

// Deterministic block sums of two values (fixed butterflies, then warp 0 over
// the warps); sh holds 64 floats.  The results in every thread.
__device__ float2 block_sum2(float a, float b, float* sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    __syncthreads();
    if (lane == 0) {
        sh[wid] = a;
        sh[32 + wid] = b;
    }
    __syncthreads();
    if (wid == 0) {
        float x = lane < nw ? sh[lane] : 0.f, y = lane < nw ? sh[32 + lane] : 0.f;
        x = warp_sum(x);
        y = warp_sum(y);
        if (lane == 0) {
            sh[0] = x;
            sh[32] = y;
        }
    }
    __syncthreads();
    return make_float2(sh[0], sh[32]);
}

__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Every thread of every CTA of the cluster; shared-memory writes before it are
// visible to the cluster after it.
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The two halves of a cluster barrier that orders nothing but the CTAs'
// start: after the wait every CTA of the cluster is running, so its shared
// memory may be written.
__device__ __forceinline__ void cluster_arrive_start()
{
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_start()
{
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
}

// Writable counterpart of `local` in cluster CTA `rank` (plain stores through
// it; the next cluster barrier publishes them).
__device__ __forceinline__ float* cluster_peer_w(float* local, unsigned rank)
{
    uint64_t remote;
    asm("mapa.u64 %0, %1, %2;" : "=l"(remote) : "l"(reinterpret_cast<uint64_t>(local)), "r"(rank));
    return reinterpret_cast<float*>(remote);
}

// shift: the first update of a step -- mu_old is the shifted mean (Alg. 1's
// shift, read as in the rollout before it; see Problem::shift_view), written back
// whole even when the iteration is degenerate, and the step's status starts at 0.
__device__ __forceinline__ void update_cluster(const Problem& pb, const float* __restrict__ C,
                                               const float* __restrict__ u, float* __restrict__ weights_out,
                                               StepState* st, float* __restrict__ cmd_out, int finalize, int shift,
                                               float* __restrict__ host_cmd = nullptr,
                                               StepState* host_st = nullptr)
{
    extern __shared__ __align__(16) float s_w[];  // N weights, then N costs
    __shared__ float s_red[64];
    __shared__ int s_redi[32];
    __shared__ float s_grp[kUpdateThreads];           // the groups' column sums, [group][column]
    __shared__ float s_mu[kUpdMaxCols];               // the new mean of this CTA's columns
    __shared__ float s_dev[kUpdMaxCols];              // their squared deviations
    __shared__ float s_jdev[kUpdCluster][kMaxDof];    // rank 0: every CTA's per-joint deviation sums
    __shared__ float s_cmd[kMaxDof];                  // rank 0: the new mean's first row
    const int N = pb.N, d = pb.d, H = pb.H, O = H * d;
    float* s_cost = s_w + ((N + 3) & ~3);
    const int tid = threadIdx.x, T = blockDim.x;
    const unsigned rank = cluster_rank();
    cluster_arrive_start();  // (waited for before the first write to a peer)
    const int cpc = (O + kUpdCluster - 1) / kUpdCluster;  // columns per CTA
    const int c0 = min(O, static_cast<int>(rank) * cpc), c1 = min(O, c0 + cpc);
    const int G = T / cpc;  // particle groups per column
    const int cl = tid % cpc, g = tid / cpc, k = c0 + cl;
    const bool col = g < G && k < c1;
    const bool lead = tid < cpc && k < c1;  // group 0 of a column: forms its totals
    // (costs, controls and the mean through L2: under a dependent launch this
    // CTA may have started before the rollout that wrote them finished)
    const int mu_off = (shift && st->step > 0) ? d : 0;
    const float mu_k = col ? (k + mu_off < O ? __ldcg(pb.mu + k + mu_off) : 0.f) : 0.f;  // mean before the update
    if (shift && rank == 0 && tid == 0) st->status = 0;
    // the costs first (the argmin waits on them), kUpdCostRegs per thread
    float cr[kUpdCostRegs];
#pragma unroll
    for (int r = 0; r < kUpdCostRegs; ++r) cr[r] = tid + r * T < N ? __ldcg(C + tid + r * T) : INFINITY;
    // this thread's particles g, g + G, ... of its column: the first kUpdBatch
    // of them are loaded now, while the weights are formed
    const int cnt = col ? (N - g + G - 1) / G : 0;
    const float* up = u + static_cast<size_t>(col ? g : 0) * O + (col ? k : 0);
    const size_t stride = static_cast<size_t>(G) * O;
    float x[kUpdBatch];
#pragma unroll
    for (int q = 0; q < kUpdBatch; ++q) x[q] = q < cnt ? up[q * stride] : 0.f;
    float wv[kUpdBatch];  // the same particles' weights
    const float* wp = s_w + g;

    // ---- min finite cost and its lowest index
    float bv = INFINITY;
    int bi = INT_MAX;
    auto visit = [&](int n, float c) {
        s_cost[n] = c;
        if (isfinite(c) && c < bv) {
            bv = c;
            bi = n;
        }
    };
#pragma unroll
    for (int r = 0; r < kUpdCostRegs; ++r)
        if (tid + r * T < N) visit(tid + r * T, cr[r]);
    for (int n = tid + kUpdCostRegs * T; n < N; n += T) visit(n, __ldcg(C + n));
    block_argmin(bv, bi, s_red, s_redi);  // (its barriers also publish s_cost)
    const float m = bv;
    const int arg = bi;
    const bool degenerate = (arg == INT_MAX);

    auto weight = [&](int n, float c) {  // Eq. 6
        if (!isfinite(c)) return 0.f;
        return pb.beta > 0.f ? expf(-(c - m) / pb.beta) : (n == arg ? 1.f : 0.f);
    };
    float s = 1.f, inv_s = 1.f, swc = 0.f;
    if (!degenerate) {
        // ---- all N weights (Eq. 6) and their sums, the same in every CTA
        float ls = 0.f, lsc = 0.f;
        for (int n = tid; n < N; n += T) {
            const float w = weight(n, s_cost[n]);
            s_w[n] = w;
            ls += w;
            if (w > 0.f) lsc = fmaf(w, s_cost[n], lsc);
        }
        const float2 sums = block_sum2(ls, lsc, s_red);  // (its barriers also publish s_w)
        s = sums.x;
        swc = sums.y;
        inv_s = 1.f / s;

        // ---- pass 1: the column's sum w (u - mu_old) over the group's particles in order
        float a1 = 0.f;
        for (int q0 = 0; q0 < cnt; q0 += kUpdBatch) {
            if (q0 > 0) {
#pragma unroll
                for (int q = 0; q < kUpdBatch; ++q) x[q] = q0 + q < cnt ? up[(q0 + q) * stride] : 0.f;
            }
#pragma unroll
            for (int q = 0; q < kUpdBatch; ++q) wv[q] = q0 + q < cnt ? wp[(q0 + q) * G] : 0.f;
#pragma unroll
            for (int q = 0; q < kUpdBatch; ++q)
                if (q0 + q < cnt) a1 = fmaf(wv[q], x[q] - mu_k, a1);
        }
        if (g < G) s_grp[tid] = a1;  // [g][cl]
        __syncthreads();
        if (lead) {  // the groups in order: the new mean, Eq. 4 (unrolled: the loads issue ahead of the sum)
            float A1 = 0.f;
#pragma unroll 6
            for (int q = 0; q < G; ++q) A1 += s_grp[q * cpc + tid];
            s_mu[tid] = fmaf(pb.alpha_mu * A1, inv_s, mu_k);
        }
        __syncthreads();

        // ---- pass 2: the column's sum w (u - mu_new)^2, Eq. 5
        const float mk = col ? s_mu[cl] : 0.f;
        float a2 = 0.f;
        for (int q0 = 0; q0 < cnt; q0 += kUpdBatch) {
            if (cnt > kUpdBatch) {  // more than one batch: x and wv hold the last one
#pragma unroll
                for (int q = 0; q < kUpdBatch; ++q) x[q] = q0 + q < cnt ? up[(q0 + q) * stride] : 0.f;
#pragma unroll
                for (int q = 0; q < kUpdBatch; ++q) wv[q] = q0 + q < cnt ? wp[(q0 + q) * G] : 0.f;
            }
#pragma unroll
            for (int q = 0; q < kUpdBatch; ++q) {
                if (q0 + q < cnt) {
                    const float e = x[q] - mk;
                    a2 = fmaf(wv[q] * e, e, a2);
                }
            }
        }
        if (g < G) s_grp[tid] = a2;  // (every pass-1 read of s_grp is behind the barrier above)
        __syncthreads();
        if (lead) {
            float A2 = 0.f;
#pragma unroll 6
            for (int q = 0; q < G; ++q) A2 += s_grp[q * cpc + tid];
            s_dev[tid] = A2;
        }
        __syncthreads();
        cluster_wait_start();
        if (tid < d) {  // joint tid's deviation over this CTA's columns, in h order, into rank 0
            float P = 0.f;
            for (int c = ((tid - c0 % d) % d + d) % d; c < c1 - c0; c += d) P += s_dev[c];
            *cluster_peer_w(&s_jdev[rank][tid], 0) = P;
        }
        if (finalize && lead && k < d) *cluster_peer_w(&s_cmd[k], 0) = s_mu[tid];
    } else {
        cluster_wait_start();
        if (finalize && lead && k < d) *cluster_peer_w(&s_cmd[k], 0) = mu_k;  // the (shifted) mean kept
    }
    cluster_barrier();  // every CTA has read the old mean; rank 0 holds the per-joint sums
    // ---- every CTA: its columns of the mean (the shifted old mean, kept, when
    // the first iteration of a step is degenerate)
    if (lead) {
        if (!degenerate)
            pb.mu[k] = s_mu[tid];
        else if (mu_off)
            pb.mu[k] = mu_k;
    }
    if (rank != 0) return;
    // ---- rank 0: sigma (Eq. 5) from the cluster's per-joint sums, in rank order
    if (degenerate) {
        if (tid == 0) {
            st->status |= STORM_WARN_DEGENERATE;
            st->best = INFINITY;
            st->wmean = INFINITY;
        }
        if (weights_out)
            for (int n = tid; n < N; n += T) weights_out[n] = 0.f;
    } else {
        if (weights_out)
            for (int n = tid; n < N; n += T) weights_out[n] = s_w[n] * inv_s;
        if (tid < d) {
            const int j = tid;
            float v = 0.f;
#pragma unroll
            for (int r = 0; r < kUpdCluster; ++r) v += s_jdev[r][j];
            v = v * inv_s / static_cast<float>(H);
            const float sg = __ldcg(pb.sigma + j);
            float var = (1.f - pb.alpha_sigma) * sg * sg + pb.alpha_sigma * v;
            var = fmaxf(var, pb.sigma_min * pb.sigma_min);
            pb.sigma[j] = sqrtf(var);
        }
        if (tid == 0) {
            st->best = m;
            st->wmean = swc / s;
        }
    }
    if (finalize) {
        if (tid < d) cmd_out[tid] = s_cmd[tid];
        if (tid == 0) st->step += 1;
        // the step's outputs straight into pinned host memory as well (host
        // calls: no device-to-host copy after the kernel), the step counter
        // last: the host returns once it sees it change
        if (host_cmd && tid == 0) {
            for (int j = 0; j < d; ++j) host_cmd[j] = s_cmd[j];
            host_st->status = st->status;
            host_st->best = st->best;
            host_st->wmean = st->wmean;
            // the counter last, as a release at system scope: the host sees the
            // outputs above once it sees the counter change
            asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(&host_st->step), "r"(st->step) : "memory");
        }
    }
}

__global__ void __cluster_dims__(kUpdCluster, 1, 1) __launch_bounds__(kUpdateThreads)
k_update(Problem pb, const float* __restrict__ C, const float* __restrict__ u,
         float* __restrict__ weights_out, StepState* st, float* __restrict__ cmd_out, int finalize, int shift,
         float* __restrict__ host_cmd, StepState* host_st)
{
    pdl_trigger();
    pdl_wait();
    update_cluster(pb, C, u, weights_out, st, cmd_out, finalize, shift, host_cmd, host_st);
}

#include "storm_adjoint.cuh"
#include "storm_mlp.cuh"
#include "storm_rollout_mlp.cuh"

// Raw noise of sample_controls: one thread per Philox block (4 values).
__global__ void k_noise(Problem pb, uint32_t step, int iter, float* __restrict__ eps)
{
    const uint32_t total = static_cast<uint32_t>(pb.N) * pb.S * pb.d;
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (4 * b >= total) return;
    if (pb.sampler == STORM_SAMPLER_HALTON) {
        for (uint32_t e = 4 * b; e < min(4 * b + 4, total); ++e) eps[e] = pb.halton[e];
        return;
    }
    const uint4 x = philox4x32_10(make_uint4(b, step, (pb.instance << 8) | static_cast<uint32_t>(iter), 0u),
                                  pb.seed_lo, pb.seed_hi);
    const float2 z01 = gauss_pair(x.x, x.y);
    const float2 z23 = gauss_pair(x.z, x.w);
    const float z[4] = {z01.x, z01.y, z23.x, z23.y};
#pragma unroll
    for (int l = 0; l < 4; ++l)
        if (4 * b + l < total) eps[4 * b + l] = z[l];
}

// The raw Philox4x32-10 words behind that noise: block first + i of the noise
// stream of (step, iter), four words per block.
__global__ void k_philox_words(Problem pb, uint32_t step, int iter, uint32_t first, int count,
                               uint32_t* __restrict__ words)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint4 x = philox4x32_10(make_uint4(first + static_cast<uint32_t>(i), step,
                                             (pb.instance << 8) | static_cast<uint32_t>(iter), 0u),
                                  pb.seed_lo, pb.seed_hi);
    reinterpret_cast<uint4*>(words)[i] = x;
}

// shift (Algorithm 1): mu_h <- mu_{h+1}, mu_{H-1} <- 0.  As the first node of a
// step it also clears the step status and skips the shift at step 0.
__device__ __forceinline__ void shift_body(const Problem& pb, StepState* st, int force)
{
    const int O = pb.H * pb.d, d = pb.d;
    const bool do_shift = force || st->step > 0;
    float v[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int o = threadIdx.x + r * blockDim.x;
        v[r] = (o + d < O) ? pb.mu[o + d] : 0.f;
    }
    __syncthreads();
    if (do_shift) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int o = threadIdx.x + r * blockDim.x;
            if (o < O) pb.mu[o] = v[r];
        }
    }
    if (threadIdx.x == 0 && !force) st->status = 0;
}

__global__ void k_shift(Problem pb, StepState* st, int force)
{
    pdl_trigger();
    shift_body(pb, st, force);
}

// Batched forward kinematics (Eq. 8): one thread per configuration.
__global__ void k_fk(Problem pb, const float* __restrict__ theta, int count, float* __restrict__ ee)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float R[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
    float p[3] = {0.f, 0.f, 0.f};
    for (int j = 0; j < pb.d; ++j) {
        const float* dh = pb.dhx + j * 8;
        dh_step(R, p, dh[0], dh[1], dh[2], dh[3], theta[static_cast<size_t>(i) * pb.d + j] + dh[4]);
    }
    float* e = ee + static_cast<size_t>(i) * 12;
    for (int r = 0; r < 3; ++r) {
        e[r * 4 + 0] = R[r * 3 + 0];
        e[r * 4 + 1] = R[r * 3 + 1];
        e[r * 4 + 2] = R[r * 3 + 2];
        e[r * 4 + 3] = p[r];
    }
}

// End-effector velocity and acceleration (Eq. 8) of count configurations.
__global__ void k_ee_twist(Problem pb, const float* __restrict__ theta, const float* __restrict__ theta_dot,
                           const float* __restrict__ theta_ddot, int count, float* __restrict__ xd_out,
                           float* __restrict__ xdd_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int d = pb.d;
    const size_t o = static_cast<size_t>(i) * d;
    float R[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
    float p[3] = {0.f, 0.f, 0.f};
    float zc[kMaxDof][3], oc[kMaxDof][3], thd[kMaxDof], thdd[kMaxDof];
#pragma unroll
    for (int j = 0; j < kMaxDof; ++j) {
        if (j < d) {
            const float* dh = pb.dhx + j * 8;
            dh_step(R, p, dh[0], dh[1], dh[2], dh[3], theta[o + j] + dh[4]);
            zc[j][0] = R[2], zc[j][1] = R[5], zc[j][2] = R[8];
            oc[j][0] = p[0], oc[j][1] = p[1], oc[j][2] = p[2];
            thd[j] = theta_dot[o + j];
            thdd[j] = theta_ddot[o + j];
        } else {
            zc[j][0] = zc[j][1] = zc[j][2] = oc[j][0] = oc[j][1] = oc[j][2] = thd[j] = thdd[j] = 0.f;
        }
    }
    float xd[6], xdd[6];
    ee_twist(zc, oc, p, thd, thdd, d, xd, xdd);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        xd_out[static_cast<size_t>(i) * 6 + k] = xd[k];
        xdd_out[static_cast<size_t>(i) * 6 + k] = xdd[k];
    }
}

// ---------------------------------------------------------------- set-up tables

__device__ double clamped_knot(int i, int S)
{
    if (i <= 3) return 0.0;
    if (i >= S) return 1.0;
    return static_cast<double>(i - 3) / static_cast<double>(S - 3);
}

// Non-zero cubic basis functions at x by the triangular (de Boor) scheme,
// scattered into a full row of S values.
__device__ void bspline_row(int S, double x, float* row)
{
    int span = S - 1;
    if (x < 1.0)
        for (int k = 3; k < S; ++k)
            if (clamped_knot(k, S) <= x && x < clamped_knot(k + 1, S)) {
                span = k;
                break;
            }
    double Nb[4], left[4], right[4];
    Nb[0] = 1.0;
    for (int j = 1; j <= 3; ++j) {
        left[j] = x - clamped_knot(span + 1 - j, S);
        right[j] = clamped_knot(span + j, S) - x;
        double saved = 0.0;
        for (int r = 0; r < j; ++r) {
            const double t = Nb[r] / (right[r + 1] + left[j - r]);
            Nb[r] = saved + right[r + 1] * t;
            saved = left[j - r] * t;
        }
        Nb[j] = saved;
    }
    for (int s = 0; s < S; ++s) row[s] = 0.f;
    for (int i = 0; i <= 3; ++i) row[span - 3 + i] = static_cast<float>(Nb[i]);
}

struct InitArgs {
    const double* dh;     // d x 4
    const double* q_min;  // d
    const double* q_max;  // d
    const double* dt;     // H
    double k_jl, qdd_max, gamma;
};

__global__ void k_init_tables(Problem pb, InitArgs a)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    float* dhx = const_cast<float*>(pb.dhx);
    for (int i = tid; i < pb.d; i += nt) {
        dhx[i * 8 + 0] = static_cast<float>(a.dh[i * 4 + 0]);
        dhx[i * 8 + 1] = static_cast<float>(cos(a.dh[i * 4 + 1]));
        dhx[i * 8 + 2] = static_cast<float>(sin(a.dh[i * 4 + 1]));
        dhx[i * 8 + 3] = static_cast<float>(a.dh[i * 4 + 2]);
        dhx[i * 8 + 4] = static_cast<float>(a.dh[i * 4 + 3]);
        dhx[i * 8 + 5] = dhx[i * 8 + 6] = dhx[i * 8 + 7] = 0.f;
        const double range = a.q_max[i] - a.q_min[i];
        const_cast<float*>(pb.qlo)[i] = static_cast<float>(a.q_min[i] + a.k_jl * range);
        const_cast<float*>(pb.qhi)[i] = static_cast<float>(a.q_max[i] - a.k_jl * range);
    }
    for (int h = tid; h < pb.H; h += nt) {
        const_cast<float*>(pb.dt)[h] = static_cast<float>(a.dt[h]);
        const_cast<float*>(pb.gpow)[h] = static_cast<float>(pow(a.gamma, static_cast<double>(h)));
        double rest = 0.0;  // (S_u(1) qdd_max dt)_h
        for (int k = pb.H - 1; k >= h; --k) rest += a.dt[k];
        const_cast<float*>(pb.vmax)[h] = static_cast<float>(a.qdd_max * rest);
        if (pb.nk > 0) {
            const double x = pb.H > 1 ? static_cast<double>(h) / (pb.H - 1) : 0.0;
            bspline_row(pb.nk, x, const_cast<float*>(pb.basis) + h * pb.nk);
        }
    }
}

// prime[k] = k-th prime (prime[0] = 2), one thread per dimension.
__global__ void k_primes(int D, int* prime)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= D) return;
    int count = -1;
    for (int c = 2;; ++c) {
        bool is_p = true;
        for (int q = 2; q * q <= c; ++q)
            if (c % q == 0) {
                is_p = false;
                break;
            }
        if (is_p && ++count == k) {
            prime[k] = c;
            return;
        }
    }
}

// Halton noise: point n+1, dimension s*d+j, radical inverse as the exact
// fraction (digit-reversed numerator) / base^digits, mapped through the
// standard normal quantile.
// Halton table (Sec. 4.3): point n + 1 in the first S*d prime bases, through
// the inverse normal CDF.  With `scramble` each digit a of dimension dim (base
// b) becomes (f a) mod b, f = 1 + (Philox4x32-10 of counter (dim, 0, 0, 3),
// first word) mod (b - 1): linearly scrambled (generalised) Halton points.
__global__ void k_halton(int N, int S, int d, const int* prime, int scramble, uint32_t seed_lo, uint32_t seed_hi,
                         float* out)
{
    const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const size_t total = static_cast<size_t>(N) * S * d;
    if (i >= total) return;
    const int dim = static_cast<int>(i % (static_cast<size_t>(S) * d));
    const uint64_t n = i / (static_cast<size_t>(S) * d) + 1;
    const uint64_t b = static_cast<uint64_t>(prime[dim]);
    uint64_t f = 1;
    if (scramble && b > 2)
        f = 1 + philox4x32_10(make_uint4(static_cast<uint32_t>(dim), 0u, 0u, 3u), seed_lo, seed_hi).x % (b - 1);
    uint64_t num = 0, den = 1, k = n;
    while (k > 0) {
        num = num * b + (f * (k % b)) % b;
        den *= b;
        k /= b;
    }
    out[i] = static_cast<float>(normcdfinv(static_cast<double>(num) / static_cast<double>(den)));
}

// ============================================================================ batched instances

// One controller of a batch, as the batched kernels see it (device memory).
struct BatchInstance {
    Problem pb;
    float* u;             // N x H x d
    float* C;             // N
    const float* state;   // 3 x d
    const float* goal;    // 7
    float* cmd;           // d
    StepState* st;
    int K;
    int pad[3];
};

struct BatchTile {
    int inst, n0, np, pad;
};

__device__ __forceinline__ void load_problem(const Problem& src, Problem& dst)
{
    const int* a = reinterpret_cast<const int*>(&src);
    int* b = reinterpret_cast<int*>(&dst);
    for (int k = threadIdx.x; k < static_cast<int>(sizeof(Problem) / 4); k += blockDim.x) b[k] = a[k];
    __syncthreads();
}

__global__ void __launch_bounds__(128) k_shift_batch(const BatchInstance* __restrict__ insts)
{
    __shared__ Problem s_pb;
    const BatchInstance& I = insts[blockIdx.x];
    load_problem(I.pb, s_pb);
    shift_body(s_pb, I.st, 0);
}

// Rollout tiles of every instance; persistent CTAs stride over the tile list
// (sorted by decreasing work, so the stride deals the big tiles first).
__global__ void __launch_bounds__(kMaxThreads)
k_rollout_batch(const BatchInstance* __restrict__ insts, const BatchTile* __restrict__ tiles,
                int n_tiles, int iter)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Problem s_pb;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const BatchTile tile = tiles[t];
        const BatchInstance& I = insts[tile.inst];
        if (iter >= I.K) continue;
        load_problem(I.pb, s_pb);
        RolloutOut out{I.u, nullptr, nullptr, nullptr, nullptr, nullptr, I.C};
        rollout_particles(s_pb, out, I.state, I.goal, I.st->step, iter, tile.n0, tile.np, smem);
        __syncthreads();
    }
}

// Rollout of every instance on the warp mapping: each warp takes (instance,
// particle group) tasks from the list (sorted by decreasing work), copies the
// instance's Problem into its own shared slot and runs the single-handle warp
// body, so each instance's results are bitwise those of its own handle
// (kFull: the full instantiation, where an instance needs it).
template <bool kFull>
__global__ void __launch_bounds__(kWarpMaxWarps * 32, 1)
k_rollout_warp_batch(const BatchInstance* __restrict__ insts, const int2* __restrict__ tasks, int n_tasks,
                     int iter, int warp_floats)
{
    extern __shared__ __align__(16) float wsm[];
    __shared__ Problem s_pb[kWarpMaxWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    Problem& pb = s_pb[warp];
    int* dst = reinterpret_cast<int*>(&pb);
    int loaded = -1;
    for (int t = blockIdx.x * wpc + warp; t < n_tasks; t += gridDim.x * wpc) {
        const int2 task = tasks[t];
        const BatchInstance& I = insts[task.x];
        if (iter >= I.K) continue;
        if (task.x != loaded) {
            __syncwarp();
            const int* src = reinterpret_cast<const int*>(&I.pb);
            for (int k = lane; k < static_cast<int>(sizeof(Problem) / 4); k += 32) dst[k] = src[k];
            __syncwarp();
            loaded = task.x;
        }
        const RolloutOut out{I.u, nullptr, nullptr, nullptr, nullptr, nullptr, I.C};
        rollout_warp_body<1, kFull>(pb, out, I.state, I.goal, I.st->step, iter, task.y, warp,
                                 wsm + size_t(warp) * warp_floats);
        __syncwarp();
    }
}

// Distribution update of every instance: cluster i (CTAs 8 i .. 8 i + 7) runs
// the single-handle update of instance i.
__global__ void __cluster_dims__(kUpdCluster, 1, 1) __launch_bounds__(kUpdateThreads)
k_update_batch(const BatchInstance* __restrict__ insts, int iter)
{
    __shared__ Problem s_pb;
    const BatchInstance& I = insts[blockIdx.x / kUpdCluster];
    if (iter >= I.K) return;  // the whole cluster
    load_problem(I.pb, s_pb);
    update_cluster(s_pb, I.C, I.u, nullptr, I.st, I.cmd, iter == I.K - 1, 0);
}

// ============================================================================ surrogate network host side

// Activations of the surrogate network for up to `cap` rows.
struct MlpBuffers {
    int cap = 0;
    bool train = false;
    __nv_bfloat16 *x = nullptr, *xT = nullptr, *a1 = nullptr, *a1T = nullptr, *a2 = nullptr,
                  *a2T = nullptr, *a3 = nullptr, *d3 = nullptr, *d3T = nullptr, *d2 = nullptr,
                  *d2T = nullptr, *d1T = nullptr;
    float *y = nullptr, *dy = nullptr, *loss_part = nullptr;
    float* part = nullptr;  // split-K partial weight gradients, kSplitMax x 256 x 256
};

struct storm_mlp {
    MlpArch a = mlp_arch(0, kMlpHid, kMlpHid, kMlpHid);
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
    __nv_bfloat16 *w1 = nullptr, *w2 = nullptr, *w2t = nullptr, *w3 = nullptr, *w3t = nullptr;
    __nv_bfloat16 *w1p = nullptr, *w2p = nullptr, *w3p = nullptr;  // packed blocks (tc::MlpView)
    MlpBuffers buf;
    float *th_b = nullptr, *t_b = nullptr, *loss_hist = nullptr;
    int* idx = nullptr;
    int cap_batch = 0, cap_idx = 0, cap_hist = 0;
    int* err = nullptr;
    int t = 0;
    int sms = 1;  // SMs of the device: the grid of the fused forward
    std::string msg = "no error";
};

void mlp_free_buffers(MlpBuffers& b)
{
    __nv_bfloat16* bf[] = {b.x, b.xT, b.a1, b.a1T, b.a2, b.a2T, b.a3, b.d3, b.d3T, b.d2, b.d2T, b.d1T};
    for (auto* q : bf)
        if (q) cudaFree(q);
    float* fl[] = {b.y, b.dy, b.loss_part, b.part};
    for (auto* q : fl)
        if (q) cudaFree(q);
    b = MlpBuffers{};
}

cudaError_t mlp_reserve(MlpBuffers& b, int rows, bool train)
{
    if (rows <= b.cap && (b.train || !train)) return cudaSuccess;
    mlp_free_buffers(b);
    const size_t R = static_cast<size_t>(rows);
    const size_t h = sizeof(__nv_bfloat16) * R * kMlpHid;
    cudaError_t e = cudaSuccess;
    auto get = [&](auto** q, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(q), bytes);
    };
    get(&b.x, sizeof(__nv_bfloat16) * R * kMlpIn);
    get(&b.a1, h);
    get(&b.a2, h);
    get(&b.y, sizeof(float) * R);
    if (train) {
        get(&b.xT, sizeof(__nv_bfloat16) * R * kMlpIn);
        get(&b.a1T, h);
        get(&b.a2T, h);
        get(&b.a3, h);
        get(&b.d3, h);
        get(&b.d3T, h);
        get(&b.d2, h);
        get(&b.d2T, h);
        get(&b.d1T, h);
        get(&b.dy, sizeof(float) * R);
        get(&b.loss_part, sizeof(float) * R);
        get(&b.part, sizeof(float) * kSplitMax * kMlpHid * kMlpHid);
    }
    if (e == cudaSuccess) {
        b.cap = rows;
        b.train = train;
    }
    return e;
}

// Split-K count for a weight gradient over R rows: a divisor of R / 128 of at
// most kSplitMax, so that every split covers whole 128-row blocks.
int split_count(int R)
{
    int sp = std::min(kSplitMax, R / tc::kBM);
    while (sp > 1 && (R / tc::kBM) % sp) --sp;
    return std::max(sp, 1);
}

// out[i] = sum over s of part[s * n + i], in the order s = 0, 1, ...; with
// tr_rows > 0 the partials are the transpose (tr_cols x tr_rows) of out
// (tr_rows x tr_cols): out[r * tr_cols + c] = sum_s part[s][c * tr_rows + r].
__global__ void k_splitk_reduce(const float* __restrict__ part, int splits, int n, int tr_rows, int tr_cols,
                                float* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int src = tr_rows > 0 ? (i % tr_cols) * tr_rows + i / tr_cols : i;
    float acc = 0.f;
    for (int s = 0; s < splits; ++s) acc += part[static_cast<size_t>(s) * n + src];
    out[i] = acc;
}

template <int BN>
cudaError_t gemm(const tc::GemmArgs& g, cudaStream_t s, int splits = 1)
{
    static int attr_set = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_set != dev) {
        const cudaError_t e = cudaFuncSetAttribute(tc::k_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   static_cast<int>(tc::gemm_smem<BN>()));
        if (e != cudaSuccess) return e;
        attr_set = dev;
    }
    if (g.M % tc::kBM || g.N != BN || g.K % 16 || g.K <= 0 || splits < 1) return cudaErrorInvalidValue;
    tc::k_gemm<BN><<<dim3(g.M / tc::kBM, splits), tc::kThreads, tc::gemm_smem<BN>(), s>>>(g);
    return cudaGetLastError();
}

// cuTensorMapEncodeTiled, reached through the runtime's driver entry point
// (the library does not link the driver library itself).
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_tiled()
{
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

// Tensor map of a rows x cols BF16 matrix (row pitch ld elements) for boxes of
// box_cols x box_rows, with or without the 128-byte shared-memory swizzle.
cudaError_t bf16_map(CUtensorMap* m, const void* base, int rows, int cols, int ld, int box_cols, int box_rows,
                     bool swizzle128)
{
    const EncodeTiled enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 2};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows)};
    const cuuint32_t step[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, step,
                           CU_TENSOR_MAP_INTERLEAVE_NONE,
                           swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Layer with the weights resident in shared memory: N = 64, 128 or 256 and
// K = 16, 64, 128 or 256.
template <int BN>
cudaError_t gemm_rw_bn(const tc::GemmArgs& g, cudaStream_t s)
{
    static int attr_dev = -1;
    static int sms = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(tc::k_gemm_ws<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(tc::gemm_ws_smem(256, 256)));
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    const int grid = std::min(g.M / tc::kBM, sms);
    // persistent: one CTA per SM walks the 128-row tiles.  Each CTA holds 2 x BN
    // TMEM columns; the shared-memory request keeps at most 512 / (2 BN) CTAs
    // on an SM, so no allocation ever waits for a co-resident CTA.
    const size_t floor_smem = BN == 256 ? 116u * 1024 : (BN == 128 ? 80u * 1024 : 48u * 1024);
    const size_t smem = std::max(tc::gemm_ws_smem(BN, g.K), floor_smem);
    // the operand's TMA loads, and the epilogue's TMA stores: 64-column x 32-row
    // boxes of the output (128-byte swizzle), 32-row x 64-column boxes of its
    // transpose
    CUtensorMap map_a{}, map_b{}, map_out{}, map_outT{};
    if (g.K % tc::kKB == 0) {  // A tiles of 128 rows x 64 K and the weights' BN x 64 K blocks by TMA, 128-byte swizzle
        cudaError_t e = bf16_map(&map_a, g.A, g.M, g.K, g.lda, tc::kKB, tc::kBM, true);
        if (e == cudaSuccess) e = bf16_map(&map_b, g.B, g.N, g.K, g.ldb, tc::kKB, BN, true);
        if (e != cudaSuccess) return e;
    }
    if (g.out_bf) {
        const cudaError_t e = bf16_map(&map_out, g.out_bf, g.M, g.N, g.ldo, 64, 32, true);
        if (e != cudaSuccess) return e;
    }
    if (g.out_bfT) {
        const cudaError_t e = bf16_map(&map_outT, g.out_bfT, g.N, g.M, g.ldoT, 32, 64, false);
        if (e != cudaSuccess) return e;
    }
    tc::k_gemm_ws<BN><<<grid, tc::kThreadsWS, smem, s>>>(g, map_a, map_b, map_out, map_outT);
    return cudaGetLastError();
}

cudaError_t gemm_rw(const tc::GemmArgs& g, cudaStream_t s)
{
    if (g.M % tc::kBM || (g.K != 16 && g.K != 64 && g.K != 128 && g.K != 256)) return cudaErrorInvalidValue;
    switch (g.N) {
    case 64: return gemm_rw_bn<64>(g, s);
    case 128: return gemm_rw_bn<128>(g, s);
    case 256: return gemm_rw_bn<256>(g, s);
    default: return cudaErrorInvalidValue;
    }
}

tc::GemmArgs gemm_args(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N,
                       int K, int* err)
{
    tc::GemmArgs g{};
    g.A = A;
    g.lda = lda;
    g.B = B;
    g.ldb = ldb;
    g.M = M;
    g.N = N;
    g.K = K;
    g.err = err;
    return g;
}

// C = P^T Q over R rows (both operands stored transposed, R contiguous: P is
// M x R, Q is N x R), split into `splits` K ranges whose FP32 partials go to
// part[split][M][N].
tc::GemmArgs weight_grad(const __nv_bfloat16* PT, const __nv_bfloat16* QT, int R, int splits, int M, int N,
                         float* part, int* err)
{
    tc::GemmArgs g = gemm_args(PT, R, QT, R, M, N, R / splits, err);
    g.out_f = part;
    g.ldf = N;
    g.split_stride = static_cast<size_t>(M) * N;
    return g;
}

cudaError_t gemm_split(const tc::GemmArgs& g, cudaStream_t s, int splits)
{
    switch (g.N) {
    case 16: return gemm<16>(g, s, splits);
    case 64: return gemm<64>(g, s, splits);
    case 128: return gemm<128>(g, s, splits);
    case 256: return gemm<256>(g, s, splits);
    default: return cudaErrorInvalidValue;
    }
}

// Weight gradient dW (rows x cols) = delta^T act over R rows into out (FP32,
// row-major): split-K GEMM and fixed-order reduction; when rows is not a
// multiple of 128 the product is formed transposed (act^T delta) and the
// reduction writes it back transposed.
int weight_grad_into(const __nv_bfloat16* deltaT, const __nv_bfloat16* actT, int R, int rows, int cols,
                     float* part, float* out, int* err, cudaStream_t s)
{
    const int sp = split_count(R);
    const bool tr = rows % tc::kBM != 0;
    const tc::GemmArgs g = tr ? weight_grad(actT, deltaT, R, sp, cols, rows, part, err)
                              : weight_grad(deltaT, actT, R, sp, rows, cols, part, err);
    if (gemm_split(g, s, sp) != cudaSuccess) return STORM_ERR_CUDA;
    const int n = rows * cols;
    k_splitk_reduce<<<(n + 255) / 256, 256, 0, s>>>(part, sp, n, tr ? rows : 0, tr ? cols : 0, out);
    return cudaGetLastError() == cudaSuccess ? STORM_OK : STORM_ERR_CUDA;
}

// Forward pass for `count` configurations (rows padded to 128); y (or the
// buffers' own y when NULL) receives the predicted distances of the padded rows.  With `train` the activations the
// backward pass needs are kept.
int mlp_forward(storm_mlp* m, MlpBuffers& b, const float* theta, int count, int dof, bool train,
                float* y, cudaStream_t s)
{
    const MlpArch& A = m->a;
    const int R = (count + tc::kBM - 1) / tc::kBM * tc::kBM;
    if (mlp_reserve(b, R, train) != cudaSuccess) return STORM_ERR_OOM;
    if (!y) y = b.y;  // after the reserve, which may reallocate b.y
    k_mlp_encode<<<(R + 255) / 256, 256, 0, s>>>(theta, count, dof, R, A.enc, b.x, train ? b.xT : nullptr);
    if (cudaGetLastError() != cudaSuccess) return STORM_ERR_CUDA;
    tc::GemmArgs g = gemm_args(b.x, kMlpIn, m->w1, kMlpIn, R, A.h1, kMlpIn, m->err);
    g.relu = 1;
    g.out_bf = b.a1;
    g.ldo = A.h1;
    if (train) {
        g.out_bfT = b.a1T;
        g.ldoT = R;
    }
    if (gemm_rw(g, s) != cudaSuccess) return STORM_ERR_CUDA;
    g = gemm_args(b.a1, A.h1, m->w2, A.h1, R, A.h2, A.h1, m->err);
    g.bias = m->p + A.ob2;
    g.relu = 1;
    g.out_bf = b.a2;
    g.ldo = A.h2;
    if (train) {
        g.out_bfT = b.a2T;
        g.ldoT = R;
    }
    if (gemm_rw(g, s) != cudaSuccess) return STORM_ERR_CUDA;
    g = gemm_args(b.a2, A.h2, m->w3, A.h2, R, A.h3, A.h2, m->err);
    g.bias = m->p + A.ob3;
    g.relu = 1;
    g.head_w = m->p + A.ow4;
    g.head_b = m->p + A.ob4;
    g.head_y = y;
    if (train) {
        g.out_bf = b.a3;
        g.ldo = A.h3;
    }
    if (gemm_rw(g, s) != cudaSuccess) return STORM_ERR_CUDA;
    return STORM_OK;
}

// Backward pass of the mean squared error after a training forward pass:
// gradient into m->g, loss into *m->loss.
int mlp_backward(storm_mlp* m, MlpBuffers& b, const float* target, int count, cudaStream_t s)
{
    const MlpArch& A = m->a;
    const int R = (count + tc::kBM - 1) / tc::kBM * tc::kBM;
    k_mlp_dhead<<<R, A.h3, 0, s>>>(b.y, target, count, R, A, b.a3, m->p, b.dy, b.d3, b.d3T, b.loss_part);
    k_mlp_head_grad<<<A.h3 + 2, 256, 0, s>>>(b.dy, b.a3, R, count, A, b.loss_part, m->g, m->loss);
    if (cudaGetLastError() != cudaSuccess) return STORM_ERR_CUDA;
    // dW3 = delta3^T a2, db3 = sum delta3
    int rc = weight_grad_into(b.d3T, b.a2T, R, A.h3, A.h2, b.part, m->g + A.oW3, m->err, s);
    if (rc) return rc;
    k_mlp_rowsum<<<A.h3, 256, 0, s>>>(b.d3T, R, m->g + A.ob3);
    // delta2 = (delta3 W3) o [a2 > 0]
    tc::GemmArgs g = gemm_args(b.d3, A.h3, m->w3t, A.h3, R, A.h2, A.h3, m->err);
    g.mask = b.a2;
    g.ldm = A.h2;
    g.out_bf = b.d2;
    g.ldo = A.h2;
    g.out_bfT = b.d2T;
    g.ldoT = R;
    if (gemm_rw(g, s) != cudaSuccess) return STORM_ERR_CUDA;
    // dW2 = delta2^T a1, db2 = sum delta2
    rc = weight_grad_into(b.d2T, b.a1T, R, A.h2, A.h1, b.part, m->g + A.oW2, m->err, s);
    if (rc) return rc;
    k_mlp_rowsum<<<A.h2, 256, 0, s>>>(b.d2T, R, m->g + A.ob2);
    // delta1 = (delta2 W2) o [a1 > 0]
    g = gemm_args(b.d2, A.h2, m->w2t, A.h2, R, A.h1, A.h2, m->err);
    g.mask = b.a1;
    g.ldm = A.h1;
    g.out_bfT = b.d1T;
    g.ldoT = R;
    if (gemm_rw(g, s) != cudaSuccess) return STORM_ERR_CUDA;
    // dW1 = delta1^T x
    rc = weight_grad_into(b.d1T, b.xT, R, A.h1, kMlpIn, b.part, m->g + A.oW1, m->err, s);
    if (rc) return rc;
    return cudaGetLastError() == cudaSuccess ? STORM_OK : STORM_ERR_CUDA;
}

int mlp_cast(storm_mlp* m, cudaStream_t s)
{
    const MlpArch& A = m->a;
    const int n = std::max(A.h1 * kMlpIn, std::max(A.h2 * A.h1, A.h3 * A.h2));
    k_mlp_cast<<<(n + 255) / 256, 256, 0, s>>>(m->p, A, m->w1, m->w2, m->w2t, m->w3, m->w3t);
    k_mlp_pack<<<(n + 255) / 256, 256, 0, s>>>(m->w1, m->w2, m->w3, A.h1, A.h2, A.h3, m->w1p, m->w2p, m->w3p);
    return cudaGetLastError() == cudaSuccess ? STORM_OK : STORM_ERR_CUDA;
}

// The network as the fused kernels read it.
tc::MlpView mlp_view(const storm_mlp* m)
{
    const MlpArch& A = m->a;
    return tc::MlpView{m->w1p, m->w2p, m->w3p, m->p + A.ob2, m->p + A.ob3, m->p + A.ow4, m->p + A.ob4,
                       A.enc, A.h1, A.h2, A.h3, m->err};
}

// ============================================================================ host runtime

struct storm_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;
    Problem pb{};
    int K = 1;
    int n_spheres_in = 0;
    size_t rollout_smem = 0, update_smem = 0;
    int grid = 0;
    int threads = kThreads;  // rollout CTA size (CTA-wide mapping)
    int mapping = STORM_MAP_WARP_PAIR;  // rollout work mapping
    int wpc = 1;                        // warps, warp pairs or four-warp groups per CTA
    bool dep_launch = false;       // step graph: rollouts and updates as programmatic dependents
    size_t warp_smem = 0;          // its dynamic shared memory
    int warp_grid = 0;
    // device allocations
    void* d_tables = nullptr;  // one block for every table
    float* d_u = nullptr;
    float* d_C = nullptr;
    float* d_io = nullptr;     // state 3d | goal 7 | cmd d | StepState
    StepState* d_st = nullptr;
    void* d_adj = nullptr;           // adjoint sums: H*d + 1 64-bit fixed-point values, count, flag
    storm_mlp* mlp = nullptr;        // learned self-collision surrogate (not owned)
    size_t mlp_smem = 0;             // k_rollout_mlp's dynamic shared memory
    float* d_ball = nullptr;         // 8: ball position, velocity (world frame), padding
    float h_ball[8] = {};
    size_t adjoint_smem = 0;
    int grad_steps = 0;
    float grad_eta = 0.f;
    float* h_io = nullptr;     // pinned mirror of d_io
    float* h_io_dev = nullptr; // the mirror's device address
    cudaGraphExec_t g_dev = nullptr, g_host = nullptr;
    std::string err = "no error";
    std::vector<double> host_sigma_init;
    double sigma_init = 0.0;
    // capacity of the world tables
    int cap_boxes = 0, cap_wsph = 0;
};

namespace {

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            (void)cudaGetLastError(); /* do not leave the error for a later check */     \
            if (h) h->err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
            return e_ == cudaErrorMemoryAllocation ? STORM_ERR_OOM : STORM_ERR_CUDA;     \
        }                                                                                \
    } while (0)

int fail(storm_handle* h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    return code;
}

int io_state(const Problem& pb) { return 0; }
int io_goal(const Problem& pb) { return 3 * pb.d; }
int io_cmd(const Problem& pb) { return 3 * pb.d + 7; }
int io_st(const Problem& pb) { return (3 * pb.d + 7 + pb.d + 3) & ~3; }
int io_floats(const Problem& pb) { return io_st(pb) + 4; }

bool finite_all(const double* p, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// Sampler, end-effector-limit and ball fields of the problem block.
void fill_sampling(const storm_params* p, Problem& pb)
{
    pb.filter = p->filter;
    pb.nk = (p->filter != STORM_FILTER_COMB && p->n_knots > 0) ? p->n_knots : 0;
    pb.spline = pb.nk > 0;  // a basis table exists
    pb.S = (p->filter == STORM_FILTER_DEFAULT && pb.nk > 0) ? pb.nk : p->H;
    pb.n_bs = p->filter == STORM_FILTER_MIXED
                  ? static_cast<int>(std::floor(p->mix_bspline * (p->N - p->n_null) + 0.5))
                  : 0;
    for (int i = 0; i < 3; ++i) {
        pb.comb[i] = static_cast<float>(p->comb[i]);
        pb.grav[i] = static_cast<float>(p->gravity[i]);
        pb.tray[i] = static_cast<float>(p->tray_center[i]);
    }
    pb.w_ee_vel = static_cast<float>(p->w_ee_vel);
    pb.w_ee_acc = static_cast<float>(p->w_ee_acc);
    pb.ee_vel_max = static_cast<float>(p->ee_vel_max);
    pb.ee_acc_max = static_cast<float>(p->ee_acc_max);
    pb.w_ball = static_cast<float>(p->w_ball);
    pb.ball = nullptr;
}

int validate(const storm_robot* r, const storm_world* w, const storm_params* p, std::string& msg)
{
    if (!r || !w || !p) return msg = "NULL robot/world/params", STORM_ERR_INVALID_ARG;
    if (r->dof < 1 || r->dof > STORM_MAX_DOF) return msg = "dof out of range", STORM_ERR_INVALID_ARG;
    if (!r->dh || !r->q_min || !r->q_max) return msg = "NULL robot table", STORM_ERR_INVALID_ARG;
    if (!finite_all(r->dh, 4 * r->dof) || !finite_all(r->q_min, r->dof) || !finite_all(r->q_max, r->dof))
        return msg = "non-finite robot table", STORM_ERR_INVALID_ARG;
    if (r->n_spheres < 0 || r->n_spheres > STORM_MAX_SPHERES)
        return msg = "n_spheres out of range", STORM_ERR_INVALID_ARG;
    if (r->n_spheres > 0 && (!r->sphere_link || !r->spheres))
        return msg = "NULL sphere table", STORM_ERR_INVALID_ARG;
    for (int s = 0; s < r->n_spheres; ++s) {
        if (r->sphere_link[s] < 0 || r->sphere_link[s] > r->dof)
            return msg = "sphere_link out of range", STORM_ERR_INVALID_ARG;
        if (!finite_all(r->spheres + 4 * s, 4) || r->spheres[4 * s + 3] < 0)
            return msg = "bad sphere", STORM_ERR_INVALID_ARG;
    }
    if (r->n_pairs < 0 || r->n_pairs > STORM_MAX_PAIRS)
        return msg = "n_pairs out of range", STORM_ERR_INVALID_ARG;
    if (r->n_pairs > 0 && !r->pairs) return msg = "NULL pairs", STORM_ERR_INVALID_ARG;
    for (int k = 0; k < 2 * r->n_pairs; ++k)
        if (r->pairs[k] < 0 || r->pairs[k] >= r->n_spheres)
            return msg = "pair index out of range", STORM_ERR_INVALID_ARG;
    if (w->n_boxes < 0 || w->n_boxes > STORM_MAX_OBSTACLES || w->n_spheres < 0 ||
        w->n_spheres > STORM_MAX_OBSTACLES)
        return msg = "obstacle count out of range", STORM_ERR_INVALID_ARG;
    if ((w->n_boxes > 0 && !w->boxes) || (w->n_spheres > 0 && !w->spheres))
        return msg = "NULL obstacle table", STORM_ERR_INVALID_ARG;
    if (!finite_all(w->boxes, 6 * w->n_boxes) || !finite_all(w->spheres, 4 * w->n_spheres))
        return msg = "non-finite obstacle", STORM_ERR_INVALID_ARG;
    if (p->N < 1 || p->N > STORM_MAX_N) return msg = "N out of range", STORM_ERR_INVALID_ARG;
    if (p->H < 1 || p->H > STORM_MAX_H) return msg = "H out of range", STORM_ERR_INVALID_ARG;
    if (p->K < 1 || p->K > 255) return msg = "K out of range", STORM_ERR_INVALID_ARG;
    if (p->n_knots != 0 && (p->n_knots < 4 || p->n_knots > p->H || p->H < 2))
        return msg = "n_knots must be 0 or in [4, H] (H >= 2)", STORM_ERR_INVALID_ARG;
    if (p->sampler != STORM_SAMPLER_PHILOX && p->sampler != STORM_SAMPLER_HALTON)
        return msg = "bad sampler", STORM_ERR_INVALID_ARG;
    if (p->rot_mode != STORM_ROT_QUAT && p->rot_mode != STORM_ROT_FROBENIUS)
        return msg = "bad rot_mode", STORM_ERR_INVALID_ARG;
    if (p->n_null < 0 || p->n_null > p->N) return msg = "n_null out of range", STORM_ERR_INVALID_ARG;
    if (!p->dt || !finite_all(p->dt, p->H)) return msg = "bad dt", STORM_ERR_INVALID_ARG;
    if (!(p->beta >= 0) || !(p->gamma >= 0) || !(p->sigma_init >= 0) || !(p->sigma_min >= 0))
        return msg = "bad beta/gamma/sigma", STORM_ERR_INVALID_ARG;
    if (p->instance >= (1u << 24)) return msg = "instance >= 2^24", STORM_ERR_INVALID_ARG;
    if (p->grad_steps < 0 || p->grad_steps > 64 || p->K + p->grad_steps > 256 ||
        !std::isfinite(p->grad_eta))
        return msg = "bad grad_steps / grad_eta", STORM_ERR_INVALID_ARG;
    if (p->halton_scramble != 0 && p->halton_scramble != 1) return msg = "bad halton_scramble", STORM_ERR_INVALID_ARG;
    if (p->filter != STORM_FILTER_DEFAULT && p->filter != STORM_FILTER_COMB && p->filter != STORM_FILTER_MIXED)
        return msg = "bad filter", STORM_ERR_INVALID_ARG;
    if (p->filter == STORM_FILTER_MIXED && p->n_knots < 4)
        return msg = "the mixed filter needs n_knots >= 4", STORM_ERR_INVALID_ARG;
    if (!finite_all(p->comb, 3) || !(p->mix_bspline >= 0.0 && p->mix_bspline <= 1.0))
        return msg = "bad comb coefficients / mix_bspline", STORM_ERR_INVALID_ARG;
    if (!(p->w_ee_vel >= 0) || !(p->w_ee_acc >= 0) || !(p->ee_vel_max >= 0) || !(p->ee_acc_max >= 0) ||
        !std::isfinite(p->w_ee_vel + p->w_ee_acc + p->ee_vel_max + p->ee_acc_max))
        return msg = "bad end-effector limits", STORM_ERR_INVALID_ARG;
    if (!std::isfinite(p->w_ball) || !finite_all(p->gravity, 3) || !finite_all(p->tray_center, 3))
        return msg = "bad ball parameters", STORM_ERR_INVALID_ARG;
    if (p->grad_steps > 0 &&
        (p->filter != STORM_FILTER_DEFAULT || p->w_ee_vel != 0 || p->w_ee_acc != 0 || p->w_ball != 0))
        return msg = "gradient refinement needs the default filter and no ee / ball terms",
               STORM_ERR_INVALID_ARG;
    return STORM_OK;
}

// Tables live in one device block; offsets in bytes, 256-aligned.
struct TablePlan {
    size_t dhx, qlo, qhi, sph, first, pairs, pblk, lbound, lcap, boxes, wsph, dt, gpow, vmax, basis, halton,
        mu, sigma, prefix, prime, raw, total;
};

TablePlan plan_tables(const Problem& pb, int cap_boxes, int cap_wsph, int raw_doubles)
{
    TablePlan t;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 15) & ~size_t(15);
        return o;
    };
    t.dhx = take(pb.d * 8 * 4);
    t.qlo = take(pb.d * 4);
    t.qhi = take(pb.d * 4);
    t.sph = take(std::max(pb.M, 1) * 16);
    t.first = take((pb.d + 2) * 4);
    t.pairs = take(std::max(pb.P, 1) * 4);
    t.pblk = take(std::max(pb.NPB, 1) * 16);
    t.lbound = take((pb.d + 1) * 16);
    t.lcap = take((pb.d + 1) * 32);
    t.boxes = take(std::max(cap_boxes, 1) * 6 * 4);
    t.wsph = take(std::max(cap_wsph, 1) * 16);
    t.dt = take(pb.H * 4);
    t.gpow = take(pb.H * 4);
    t.vmax = take(pb.H * 4);
    t.basis = take(pb.nk > 0 ? pb.H * pb.nk * 4 : 4);
    t.prefix = off;  // dhx .. basis: what every rollout CTA copies to shared memory
    t.mu = take(pb.H * pb.d * 4);
    t.sigma = take(pb.d * 4);
    t.halton = take(pb.sampler == STORM_SAMPLER_HALTON ? size_t(pb.N) * pb.S * pb.d * 4 : 4);
    t.prime = take(pb.S * pb.d * 4);
    t.raw = take(raw_doubles * 8);
    t.total = off;
    return t;
}

int upload_world(storm_handle* h, const storm_world* w)
{
    std::vector<float> boxes(6 * std::max(w->n_boxes, 1)), ws(4 * std::max(w->n_spheres, 1));
    for (int i = 0; i < 6 * w->n_boxes; ++i) boxes[i] = static_cast<float>(w->boxes[i]);
    for (int i = 0; i < 4 * w->n_spheres; ++i) ws[i] = static_cast<float>(w->spheres[i]);
    if (w->n_boxes)
        CK(cudaMemcpyAsync(const_cast<float*>(h->pb.boxes), boxes.data(), 6 * 4 * w->n_boxes,
                           cudaMemcpyHostToDevice, h->stream));
    if (w->n_spheres)
        CK(cudaMemcpyAsync(const_cast<float4*>(h->pb.wsph), ws.data(), 16 * w->n_spheres,
                           cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->pb.B = w->n_boxes;
    h->pb.O = w->n_spheres;
    return STORM_OK;
}

// A problem the lean warp rollout does not cover (see rollout_warp_body).
bool needs_full_rollout(const Problem& pb)
{
    return pb.w_ee_vel != 0.f || pb.w_ee_acc != 0.f || (pb.ball && pb.w_ball != 0.f) ||
           pb.filter != STORM_FILTER_DEFAULT || pb.rot_mode != STORM_ROT_QUAT || pb.sampler != STORM_SAMPLER_PHILOX;
}

// Warps per particle group of a warp mapping.
int warps_per_group(int mapping)
{
    return mapping == STORM_MAP_WARP_QUAD ? 4 : mapping == STORM_MAP_WARP_PAIR ? 2 : 1;
}

// A kernel launch; with dep set, as a programmatic dependent of the stream's
// previous kernel (it may start before that kernel ends and must pdl_wait
// before reading anything the predecessor writes).
template <typename... Params, typename... Args>
cudaError_t launch_kernel(void (*kernel)(Params...), unsigned grid, unsigned block, size_t smem,
                          cudaStream_t s, bool dep, Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = dep ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// dep: launched as a dependent of the previous kernel.  Only the step graph
// sets it, where the predecessor (the shift or a non-final update) never
// advances the step counter that the rollout reads before its pdl_wait.
int launch_rollout(storm_handle* h, cudaStream_t s, const RolloutOut& out, const float* state,
                   const float* goal, int step_override, int iter, bool dep = false, bool shift = false)
{
    Problem pb = h->pb;
    pb.dep_launch = dep ? 1 : 0;
    pb.shift_view = shift ? 1 : 0;
    // the full instantiation where the problem or the call needs its extra code
    const bool full = needs_full_rollout(pb) || out.theta || out.theta_dot || out.ee || out.terms || out.cost;
    if (pb.self_mode != 0 && h->mlp) {  // the learned self collision: the network inside the rollout
        pb.dep_launch = 0;
        const WarpPlan wp = warp_plan(pb, 1);
        const int grid = (pb.N + wp.PW * kMlpWarps - 1) / (wp.PW * kMlpWarps);
        CK(launch_kernel(full ? k_rollout_mlp<true> : k_rollout_mlp<false>, grid, tc::tile_threads(kMlpEpi),
                         h->mlp_smem, s, false, pb, out, state, goal, static_cast<const StepState*>(h->d_st),
                         step_override, iter, mlp_view(h->mlp)));
        return STORM_OK;
    }
    const StepState* st = h->d_st;
    if (h->mapping == STORM_MAP_WARP)
        CK(launch_kernel(full ? k_rollout_warp<1, true> : k_rollout_warp<1, false>, h->warp_grid, h->wpc * 32,
                         h->warp_smem, s, dep, pb, out, state, goal, st, step_override, iter));
    else if (h->mapping == STORM_MAP_WARP_PAIR)
        CK(launch_kernel(full ? k_rollout_warp<2, true> : k_rollout_warp<2, false>, h->warp_grid, h->wpc * 64,
                         h->warp_smem, s, dep, pb, out, state, goal, st, step_override, iter));
    else if (h->mapping == STORM_MAP_WARP_QUAD)
        CK(launch_kernel(full ? k_rollout_warp<4, true> : k_rollout_warp<4, false>, h->warp_grid, h->wpc * 128,
                         h->warp_smem, s, dep, pb, out, state, goal, st, step_override, iter));
    else
        CK(launch_kernel(k_rollout, h->grid, h->threads, h->rollout_smem, s, dep, pb, out, state, goal,
                         static_cast<const StepState*>(h->d_st), step_override, iter));
    return STORM_OK;
}

// shift: the first update of a step graph (see update_cluster).
// host_out: also write the command and the step record into the pinned mirror
// (at the last iteration).
int launch_update(storm_handle* h, cudaStream_t s, const float* C, const float* u, float* w,
                  float* cmd, int finalize, bool dep = false, bool shift = false, bool host_out = false)
{
    float* host_cmd = host_out ? h->h_io_dev + io_cmd(h->pb) : nullptr;
    StepState* host_st = host_out ? reinterpret_cast<StepState*>(h->h_io_dev + io_st(h->pb)) : nullptr;
    CK(launch_kernel(k_update, kUpdCluster, kUpdateThreads, h->update_smem, s, dep, h->pb, C, u, w, h->d_st, cmd,
                     finalize, shift ? 1 : 0, host_cmd, host_st));
    return STORM_OK;
}

int launch_adjoint(storm_handle* h, cudaStream_t s, const float* state, const float* goal,
                   const float* mean, int step_override, int iter, float* grad, float* J, float* Ctot,
                   float eta, float* cmd, int finalize)
{
    // 128 threads: the per-(step, sphere) and per-(step, pair block) collision
    // loops split four warps' ways; at 125 registers 4 CTAs fit an SM, so the
    // paper workload's 500 particles stay one wave.  The CTA that finishes
    // last turns the fixed-point sums into grad and J (no second kernel).
    const int threads = 128;
    const int HD = h->pb.H * h->pb.d;
    AdjAcc acc{reinterpret_cast<unsigned long long*>(h->d_adj),
               reinterpret_cast<unsigned int*>(reinterpret_cast<unsigned long long*>(h->d_adj) + HD + 1),
               reinterpret_cast<int*>(reinterpret_cast<unsigned long long*>(h->d_adj) + HD + 1) + 1};
    k_adjoint<<<h->pb.N, threads, h->adjoint_smem, s>>>(h->pb, mean, state, goal, h->d_st, step_override, iter,
                                                         acc, Ctot, grad, J, eta, cmd, finalize);
    CK(cudaGetLastError());
    return STORM_OK;
}

// Enqueue the kernels of one control step (device inputs in d_io).  Alg. 1's
// shift is folded into the first iteration: its rollouts and update read the
// shifted mean and the update stores it (no kernel of its own).  host_out: the
// update that finishes the step also writes the command and the step record
// into the pinned mirror (see step_outputs_by_kernel).
int enqueue_step_kernels(storm_handle* h, cudaStream_t s, bool host_out = false)
{
    RolloutOut out{h->d_u, nullptr, nullptr, nullptr, nullptr, nullptr, h->d_C};
    const float* state = h->d_io + io_state(h->pb);
    const float* goal = h->d_io + io_goal(h->pb);
    float* cmd = h->d_io + io_cmd(h->pb);
    for (int k = 0; k < h->K; ++k) {
        int rc = launch_rollout(h, s, out, state, goal, -1, k, h->dep_launch, k == 0);
        if (rc) return rc;
        const bool last = k == h->K - 1 && h->grad_steps == 0;
        rc = launch_update(h, s, h->d_C, h->d_u, nullptr, cmd, last, h->dep_launch, k == 0, host_out && last);
        if (rc) return rc;
    }
    for (int g = 0; g < h->grad_steps; ++g) {  // gradient refinement of the mean
        int rc = launch_adjoint(h, s, state, goal, h->pb.mu, -1, h->K + g, nullptr, nullptr,
                                nullptr, h->grad_eta, cmd, g == h->grad_steps - 1);
        if (rc) return rc;
    }
    return STORM_OK;
}

// Opt every kernel with dynamic shared memory in to the device maximum, so that
// handles of different sizes never lower each other's limit.
int allow_smem(storm_handle* h)
{
    int optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    cudaFuncAttributes ra, ua, aa, wa;
    CK(cudaFuncGetAttributes(&ra, k_rollout));
    using WarpKernel = void (*)(Problem, RolloutOut, const float*, const float*, const StepState*, int, int);
    const WarpKernel warp_kernels[] = {k_rollout_warp<1, false>, k_rollout_warp<1, true>, k_rollout_warp<2, false>,
                                       k_rollout_warp<2, true>,  k_rollout_warp<4, false>, k_rollout_warp<4, true>};
    for (WarpKernel kf : warp_kernels) {
        CK(cudaFuncGetAttributes(&wa, kf));
        CK(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - static_cast<int>(wa.sharedSizeBytes)));
    }
    CK(cudaFuncGetAttributes(&ua, k_update));
    CK(cudaFuncGetAttributes(&aa, k_adjoint));
    if (h->rollout_smem + ra.sharedSizeBytes > size_t(optin) ||
        h->update_smem + ua.sharedSizeBytes > size_t(optin) ||
        h->adjoint_smem + aa.sharedSizeBytes > size_t(optin))
        return fail(h, STORM_ERR_INVALID_ARG, "problem needs more shared memory than a CTA has");
    CK(cudaFuncSetAttribute(k_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            optin - static_cast<int>(aa.sharedSizeBytes)));
    CK(cudaFuncSetAttribute(k_rollout, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            optin - static_cast<int>(ra.sharedSizeBytes)));
    CK(cudaFuncSetAttribute(k_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            optin - static_cast<int>(ua.sharedSizeBytes)));
    return STORM_OK;
}

void destroy_graphs(storm_handle* h)
{
    if (h->g_dev) cudaGraphExecDestroy(h->g_dev);
    if (h->g_host) cudaGraphExecDestroy(h->g_host);
    h->g_dev = h->g_host = nullptr;
}

constexpr uint32_t kStepPending = 0xffffffffu;  // host mirror's step field while a host call runs
constexpr int kStepPollMs = 2000;               // then the stream is synchronised instead

// The host graph's outputs (command, step record) written by the update that
// finishes the step straight into the pinned mirror, with no copy node: when
// no gradient refinement follows the last update.
bool step_outputs_by_kernel(const storm_handle* h) { return h->grad_steps == 0; }

int build_graphs(storm_handle* h)
{
    destroy_graphs(h);
    for (int with_io = 0; with_io < 2; ++with_io) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = STORM_OK;
        if (with_io) {
            const size_t in_bytes = sizeof(float) * (3 * h->pb.d + 7);
            rc = cudaMemcpyAsync(h->d_io, h->h_io, in_bytes, cudaMemcpyHostToDevice, h->cap_stream)
                     ? STORM_ERR_CUDA
                     : STORM_OK;
        }
        if (!rc) rc = enqueue_step_kernels(h, h->cap_stream, with_io && step_outputs_by_kernel(h));
        if (!rc && with_io && !step_outputs_by_kernel(h)) {
            const size_t off = io_cmd(h->pb);
            const size_t bytes = sizeof(float) * (io_floats(h->pb) - off);
            rc = cudaMemcpyAsync(h->h_io + off, h->d_io + off, bytes, cudaMemcpyDeviceToHost,
                                 h->cap_stream)
                     ? STORM_ERR_CUDA
                     : STORM_OK;
        }
        cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        CK(e);
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        CK(e);
        (with_io ? h->g_host : h->g_dev) = ex;
    }
    // upload the executable graphs once so the first replay is not slower
    CK(cudaGraphUpload(h->g_dev, h->stream));
    CK(cudaGraphUpload(h->g_host, h->stream));
    return STORM_OK;
}

void free_all(storm_handle* h)
{
    destroy_graphs(h);
    if (h->d_tables) cudaFree(h->d_tables);
    if (h->d_u) cudaFree(h->d_u);
    if (h->d_C) cudaFree(h->d_C);
    if (h->d_io) cudaFree(h->d_io);
    if (h->d_adj) cudaFree(h->d_adj);
    if (h->d_ball) cudaFree(h->d_ball);
    if (h->h_io) cudaFreeHost(h->h_io);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

// Group self-collision pairs (sorted sphere indices, a < b) by the links of
// their spheres.  A group that is exactly every sphere of one link against
// every sphere of another becomes blocks of at most 8 second-link spheres;
// anything else stays an explicit pair.
void build_pair_blocks(const std::vector<uint32_t>& pairs, const std::vector<int>& first, int d,
                       std::vector<uint4>& blocks, std::vector<uint32_t>& rest)
{
    auto link_of = [&](int s) {
        int f = 0;
        while (f < d && s >= first[f + 1]) ++f;
        return f;
    };
    std::map<std::pair<int, int>, std::vector<uint32_t>> groups;
    for (uint32_t pr : pairs) groups[{link_of(pr & 0xffff), link_of(pr >> 16)}].push_back(pr);
    for (auto& g : groups) {
        const int la = g.first.first, lb = g.first.second;
        const int na = first[la + 1] - first[la], nb = first[lb + 1] - first[lb];
        const std::set<uint32_t> uniq(g.second.begin(), g.second.end());
        const bool complete = la != lb && uniq.size() == g.second.size() &&
                              static_cast<int>(uniq.size()) == na * nb;
        if (complete) {
            for (int b0 = first[lb]; b0 < first[lb + 1]; b0 += 8)
                blocks.push_back(make_uint4(first[la], first[la + 1], b0, std::min(8, first[lb + 1] - b0)));
        } else {
            rest.insert(rest.end(), g.second.begin(), g.second.end());
        }
    }
}

// Host-side tables of one problem, before upload.
struct HostTables {
    std::vector<float> sph, boxes, wsph;
    std::vector<int> first;
    std::vector<uint32_t> pairs;
    std::vector<uint4> blocks;
    std::vector<float4> lbound;  // per frame: bounding sphere of its spheres (local)
    std::vector<float4> lcap;    // per frame: capsule of its spheres (local), two float4
    std::vector<double> raw;  // dh | q_min | q_max | dt, read by the set-up kernel
    double k_jl = 0, qdd_max = 0, gamma = 0;
    int halton_scramble = 0;
};

// Scalars of the problem and its host tables: spheres sorted by link (stable),
// pairs remapped to that order and grouped into link-pair blocks.
void fill_problem(const storm_robot* r, const storm_world* w, const storm_params* p, Problem& pb,
                  HostTables& ht)
{
    pb = Problem{};
    pb.N = p->N;
    pb.H = p->H;
    pb.d = r->dof;
    fill_sampling(p, pb);
    pb.sampler = p->sampler;
    pb.n_null = p->n_null;
    pb.rot_mode = p->rot_mode;
    pb.M = r->n_spheres;
    pb.B = w->n_boxes;
    pb.O = w->n_spheres;
    pb.beta = static_cast<float>(p->beta);
    pb.alpha_mu = static_cast<float>(p->alpha_mu);
    pb.alpha_sigma = static_cast<float>(p->alpha_sigma);
    pb.sigma_min = static_cast<float>(p->sigma_min);
    pb.w_pos = static_cast<float>(p->w_pos);
    pb.w_rot = static_cast<float>(p->w_rot);
    pb.w_stop = static_cast<float>(p->w_stop);
    pb.w_joint = static_cast<float>(p->w_joint);
    pb.w_manip = static_cast<float>(p->w_manip);
    pb.w_coll = static_cast<float>(p->w_coll);
    pb.w_smooth = static_cast<float>(p->w_smooth);
    for (int i = 0; i < 3; ++i) {
        pb.pos_w[i] = static_cast<float>(p->pos_axis_w[i]);
        pb.rot_w[i] = static_cast<float>(p->rot_axis_w[i]);
    }
    pb.k_m = static_cast<float>(p->k_m);
    pb.seed_lo = static_cast<uint32_t>(p->seed & 0xffffffffu);
    pb.seed_hi = static_cast<uint32_t>(p->seed >> 32);
    pb.instance = p->instance;
    // particles per CTA: about 64 (particle, step) items
    pb.ppc = std::max(1, std::min(pb.N, 64 / pb.H));

    std::vector<int> order(pb.M);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return r->sphere_link[a] < r->sphere_link[b]; });
    std::vector<int> rank(pb.M);
    for (int i = 0; i < pb.M; ++i) rank[order[i]] = i;
    ht.sph.assign(4 * std::max(pb.M, 1), 0.f);
    ht.first.assign(pb.d + 2, 0);
    for (int i = 0; i < pb.M; ++i) {
        for (int k = 0; k < 4; ++k) ht.sph[4 * i + k] = static_cast<float>(r->spheres[4 * order[i] + k]);
        ht.first[r->sphere_link[order[i]] + 1]++;
    }
    for (int f = 0; f <= pb.d; ++f) ht.first[f + 1] += ht.first[f];
    std::vector<uint32_t> all_pairs(r->n_pairs);
    for (int k = 0; k < r->n_pairs; ++k) {
        uint32_t a = rank[r->pairs[2 * k]], b = rank[r->pairs[2 * k + 1]];
        if (a > b) std::swap(a, b);
        all_pairs[k] = a | (b << 16);
    }
    ht.blocks.clear();
    ht.pairs.clear();
    build_pair_blocks(all_pairs, ht.first, pb.d, ht.blocks, ht.pairs);
    pb.P = static_cast<int>(ht.pairs.size());
    pb.NPB = static_cast<int>(ht.blocks.size());
    {
        // block range of every frame pair (blocks come sorted by (la, lb))
        auto link_of = [&](int sidx) {
            int f = 0;
            while (f < pb.d && sidx >= ht.first[f + 1]) ++f;
            return f;
        };
        int bk = 0;
        for (int la = 0; la < kMaxDof; ++la)
            for (int lb = la + 1; lb <= kMaxDof; ++lb) {
                const int t = link_pair_index(la, lb);
                pb.lp_begin[t] = static_cast<uint16_t>(bk);
                while (bk < pb.NPB && link_of(ht.blocks[bk].x) == la && link_of(ht.blocks[bk].z) == lb) ++bk;
            }
        pb.lp_begin[kLinkPairs] = static_cast<uint16_t>(bk);
    }
    ht.pairs.resize(std::max(pb.P, 1));
    ht.blocks.resize(std::max(pb.NPB, 1));
    // per frame: the sphere about the centroid of its spheres' centres that
    // encloses them all, padded by 1e-4 m against FP32 rounding in the tests
    ht.lbound.assign(pb.d + 1, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int f = 0; f <= pb.d; ++f) {
        const int a = ht.first[f], b = ht.first[f + 1];
        if (a == b) continue;
        double c[3] = {0, 0, 0};
        for (int i = a; i < b; ++i)
            for (int k = 0; k < 3; ++k) c[k] += ht.sph[4 * i + k] / double(b - a);
        double R = 0.0;
        for (int i = a; i < b; ++i) {
            const double dx = ht.sph[4 * i] - c[0], dy = ht.sph[4 * i + 1] - c[1], dz = ht.sph[4 * i + 2] - c[2];
            R = std::max(R, std::sqrt(dx * dx + dy * dy + dz * dz) + ht.sph[4 * i + 3]);
        }
        ht.lbound[f] = make_float4(static_cast<float>(c[0]), static_cast<float>(c[1]), static_cast<float>(c[2]),
                                   static_cast<float>(R + 1e-4));
    }
    // per frame: a capsule (the points within R of a segment) holding every
    // sphere of the frame; the segment joins the two sphere centres farthest
    // apart, R reaches the farthest sphere surface, padded by 1 mm, which covers
    // FP32 rounding in the device's segment distances (their worst case, nearly
    // parallel segments, is below 0.3 mm for links up to 1 m)
    ht.lcap.assign(2 * (pb.d + 1), make_float4(0.f, 0.f, 0.f, 0.f));
    for (int f = 0; f <= pb.d; ++f) {
        const int a = ht.first[f], b = ht.first[f + 1];
        if (a == b) continue;
        auto ctr = [&](int i, int k) { return static_cast<double>(ht.sph[4 * i + k]); };
        int e0 = a, e1 = a;
        double far = -1.0;
        for (int i = a; i < b; ++i)
            for (int j = i; j < b; ++j) {
                double d2 = 0.0;
                for (int k = 0; k < 3; ++k) d2 += (ctr(i, k) - ctr(j, k)) * (ctr(i, k) - ctr(j, k));
                if (d2 > far) far = d2, e0 = i, e1 = j;
            }
        double seg[3], len2 = 0.0;
        for (int k = 0; k < 3; ++k) seg[k] = ctr(e1, k) - ctr(e0, k), len2 += seg[k] * seg[k];
        double R = 0.0;
        for (int i = a; i < b; ++i) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += (ctr(i, k) - ctr(e0, k)) * seg[k];
            s = len2 > 0.0 ? std::min(1.0, std::max(0.0, s / len2)) : 0.0;
            double d2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double e = ctr(i, k) - (ctr(e0, k) + s * seg[k]);
                d2 += e * e;
            }
            R = std::max(R, std::sqrt(d2) + ht.sph[4 * i + 3]);
        }
        ht.lcap[2 * f] = make_float4(ht.sph[4 * e0], ht.sph[4 * e0 + 1], ht.sph[4 * e0 + 2],
                                     static_cast<float>(R + 1e-3));
        ht.lcap[2 * f + 1] = make_float4(ht.sph[4 * e1], ht.sph[4 * e1 + 1], ht.sph[4 * e1 + 2], 0.f);
    }
    pb.broadphase = 1;
    ht.boxes.assign(6 * std::max(pb.B, 1), 0.f);
    ht.wsph.assign(4 * std::max(pb.O, 1), 0.f);
    for (int i = 0; i < 6 * pb.B; ++i) ht.boxes[i] = static_cast<float>(w->boxes[i]);
    for (int i = 0; i < 4 * pb.O; ++i) ht.wsph[i] = static_cast<float>(w->spheres[i]);
    ht.raw.clear();
    ht.raw.insert(ht.raw.end(), r->dh, r->dh + 4 * pb.d);
    ht.raw.insert(ht.raw.end(), r->q_min, r->q_min + pb.d);
    ht.raw.insert(ht.raw.end(), r->q_max, r->q_max + pb.d);
    ht.raw.insert(ht.raw.end(), p->dt, p->dt + pb.H);
    ht.k_jl = p->k_jl;
    ht.halton_scramble = p->halton_scramble;
    ht.qdd_max = p->qdd_max;
    ht.gamma = p->gamma;
}

// Point the problem's tables into `base` (laid out by `t`), copy the host tables
// and enqueue the set-up kernels (derived tables, Halton noise).
cudaError_t upload_problem(Problem& pb, const HostTables& ht, char* base, const TablePlan& t,
                           cudaStream_t s)
{
    pb.dhx = reinterpret_cast<float*>(base + t.dhx);
    pb.qlo = reinterpret_cast<float*>(base + t.qlo);
    pb.qhi = reinterpret_cast<float*>(base + t.qhi);
    pb.sph = reinterpret_cast<float4*>(base + t.sph);
    pb.link_first = reinterpret_cast<int*>(base + t.first);
    pb.pairs = reinterpret_cast<uint32_t*>(base + t.pairs);
    pb.pblk = reinterpret_cast<uint4*>(base + t.pblk);
    pb.boxes = reinterpret_cast<float*>(base + t.boxes);
    pb.wsph = reinterpret_cast<float4*>(base + t.wsph);
    pb.dt = reinterpret_cast<float*>(base + t.dt);
    pb.gpow = reinterpret_cast<float*>(base + t.gpow);
    pb.vmax = reinterpret_cast<float*>(base + t.vmax);
    pb.basis = reinterpret_cast<float*>(base + t.basis);
    pb.halton = reinterpret_cast<float*>(base + t.halton);
    pb.mu = reinterpret_cast<float*>(base + t.mu);
    pb.sigma = reinterpret_cast<float*>(base + t.sigma);
    pb.tables = reinterpret_cast<const uint4*>(base);
    pb.table_bytes = static_cast<int>(t.prefix);
    int* d_prime = reinterpret_cast<int*>(base + t.prime);
    double* d_raw = reinterpret_cast<double*>(base + t.raw);
    cudaError_t e = cudaSuccess;
    auto put = [&](const void* dst, const void* src, size_t bytes) {
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(const_cast<void*>(dst), src, bytes, cudaMemcpyHostToDevice, s);
    };
    put(pb.sph, ht.sph.data(), 4 * ht.sph.size());
    put(pb.link_first, ht.first.data(), 4 * ht.first.size());
    put(pb.pairs, ht.pairs.data(), 4 * ht.pairs.size());
    put(pb.pblk, ht.blocks.data(), 16 * ht.blocks.size());
    pb.lbound = reinterpret_cast<float4*>(base + t.lbound);
    put(pb.lbound, ht.lbound.data(), 16 * ht.lbound.size());
    pb.lcap = reinterpret_cast<float4*>(base + t.lcap);
    put(pb.lcap, ht.lcap.data(), 16 * ht.lcap.size());
    put(pb.boxes, ht.boxes.data(), 4 * ht.boxes.size());
    put(pb.wsph, ht.wsph.data(), 4 * ht.wsph.size());
    put(d_raw, ht.raw.data(), 8 * ht.raw.size());
    if (e != cudaSuccess) return e;
    InitArgs ia{d_raw, d_raw + 4 * pb.d, d_raw + 5 * pb.d, d_raw + 6 * pb.d, ht.k_jl, ht.qdd_max,
                ht.gamma};
    k_init_tables<<<1, 64, 0, s>>>(pb, ia);
    if (pb.sampler == STORM_SAMPLER_HALTON) {
        const int D = pb.S * pb.d;
        k_primes<<<(D + 127) / 128, 128, 0, s>>>(D, d_prime);
        const size_t total = size_t(pb.N) * pb.S * pb.d;
        k_halton<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(
            pb.N, pb.S, pb.d, d_prime, ht.halton_scramble, pb.seed_lo, pb.seed_hi, const_cast<float*>(pb.halton));
    }
    return cudaGetLastError();
}

int create_impl(storm_handle* h, const storm_robot* r, const storm_world* w, const storm_params* p,
                void* stream)
{
    CK(cudaGetDevice(&h->device));
    if (stream) {
        h->stream = static_cast<cudaStream_t>(stream);
    } else {
        CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));

    HostTables ht;
    Problem& pb = h->pb;
    fill_problem(r, w, p, pb, ht);
    h->K = p->K;
    h->grad_steps = p->grad_steps;
    h->grad_eta = static_cast<float>(p->grad_eta);
    h->sigma_init = p->sigma_init;
    h->cap_boxes = STORM_MAX_OBSTACLES;
    h->cap_wsph = STORM_MAX_OBSTACLES;
    h->grid = (pb.N + pb.ppc - 1) / pb.ppc;
    {
        const WarpPlan wp = warp_plan(pb, warps_per_group(h->mapping));
        h->warp_smem = sizeof(float) * size_t(wp.floats) * h->wpc;
        h->warp_grid = (pb.N + wp.PW * h->wpc - 1) / (wp.PW * h->wpc);
    }

    const TablePlan t = plan_tables(pb, h->cap_boxes, h->cap_wsph, static_cast<int>(ht.raw.size()));
    CK(cudaMalloc(&h->d_tables, t.total));
    CK(cudaMalloc(&h->d_u, sizeof(float) * size_t(pb.N) * pb.H * pb.d));
    CK(cudaMalloc(&h->d_C, sizeof(float) * pb.N));
    CK(cudaMalloc(&h->d_ball, sizeof(float) * 8));
    CK(cudaMemsetAsync(h->d_ball, 0, sizeof(float) * 8, h->stream));
    pb.ball = h->d_ball;  // the ball state of storm_set_ball (zero until set)
    CK(cudaMalloc(&h->d_io, sizeof(float) * io_floats(pb)));
    CK(cudaMallocHost(&h->h_io, sizeof(float) * io_floats(pb)));
    CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&h->h_io_dev), h->h_io, 0));
    {
        const size_t adj_bytes = sizeof(unsigned long long) * (pb.H * pb.d + 2);
        CK(cudaMalloc(&h->d_adj, adj_bytes));
        CK(cudaMemsetAsync(h->d_adj, 0, adj_bytes, h->stream));
    }
    std::memset(h->h_io, 0, sizeof(float) * io_floats(pb));
    h->d_st = reinterpret_cast<StepState*>(h->d_io + io_st(pb));
    CK(cudaMemsetAsync(h->d_io, 0, sizeof(float) * io_floats(pb), h->stream));
    CK(upload_problem(pb, ht, static_cast<char*>(h->d_tables), t, h->stream));

    const RolloutLayout L = rollout_layout(pb);
    h->rollout_smem = L.bytes;
    h->update_smem = sizeof(float) * 2 * ((pb.N + 3) & ~3);
    h->adjoint_smem = adjoint_layout(pb).bytes;
    int rc = allow_smem(h);
    if (rc) return rc;
    rc = storm_reset(h);
    if (rc) return rc;
    return build_graphs(h);
}

}  // namespace

// ============================================================================ C ABI

extern "C" {

const char* storm_status_string(int s)
{
    switch (s) {
    case STORM_OK: return "ok";
    case STORM_WARN_DEGENERATE: return "warning: no finite total cost; distribution kept";
    case STORM_ERR_INVALID_ARG: return "invalid argument";
    case STORM_ERR_CUDA: return "CUDA error";
    case STORM_ERR_OOM: return "out of device memory";
    case STORM_ERR_NONFINITE: return "non-finite state or goal";
    case STORM_ERR_TIMEOUT: return "timeout";
    case STORM_ERR_STATE: return "checkpoint does not match handle";
    default: return "unknown status";
    }
}

const char* storm_last_error(const storm_handle* h) { return h ? h->err.c_str() : "NULL handle"; }

int storm_create(const storm_robot* robot, const storm_world* world, const storm_params* params,
                 void* cuda_stream, storm_handle** out)
{
    if (!out) return STORM_ERR_INVALID_ARG;
    *out = nullptr;
    std::string msg;
    const int v = validate(robot, world, params, msg);
    if (v) return v;
    storm_handle* h = new (std::nothrow) storm_handle();
    if (!h) return STORM_ERR_OOM;
    const int rc = create_impl(h, robot, world, params, cuda_stream);
    if (rc) {
        fprintf(stderr, "storm_create: %s\n", h->err.c_str());
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return STORM_OK;
}

void storm_destroy(storm_handle* h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

int storm_reset(storm_handle* h)
{
    if (!h) return STORM_ERR_INVALID_ARG;
    const int O = h->pb.H * h->pb.d;
    std::vector<float> mu(O, 0.f), sg(h->pb.d, static_cast<float>(h->sigma_init));
    CK(cudaMemcpyAsync(h->pb.mu, mu.data(), 4 * O, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->pb.sigma, sg.data(), 4 * h->pb.d, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(h->d_st, 0, sizeof(StepState), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return STORM_OK;
}

int storm_step(storm_handle* h, const float* state, const float* goal, float* cmd,
               storm_step_info* info)
{
    if (!h || !state || !goal || !cmd) return fail(h, STORM_ERR_INVALID_ARG, "NULL argument");
    const int d = h->pb.d;
    for (int i = 0; i < 3 * d; ++i)
        if (!std::isfinite(state[i])) return fail(h, STORM_ERR_NONFINITE, "non-finite state");
    for (int i = 0; i < 7; ++i)
        if (!std::isfinite(goal[i])) return fail(h, STORM_ERR_NONFINITE, "non-finite goal");
    std::memcpy(h->h_io + io_state(h->pb), state, sizeof(float) * 3 * d);
    std::memcpy(h->h_io + io_goal(h->pb), goal, sizeof(float) * 7);
    StepState* st = reinterpret_cast<StepState*>(h->h_io + io_st(h->pb));
    volatile uint32_t* st_step = &st->step;
    const bool poll = step_outputs_by_kernel(h);
    if (poll) *st_step = kStepPending;  // the last update overwrites it, last of the outputs
    CK(cudaGraphLaunch(h->g_host, h->stream));
    if (poll) {
        // wait for the outputs in pinned memory rather than for the stream to
        // drain; past a bound (or on any device error) the stream decides
        const auto t0 = std::chrono::steady_clock::now();
        while (*st_step == kStepPending) {
            if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(kStepPollMs)) break;
        }
        std::atomic_thread_fence(std::memory_order_acquire);
        if (*st_step == kStepPending) CK(cudaStreamSynchronize(h->stream));
        if (*st_step == kStepPending) return fail(h, STORM_ERR_CUDA, "step outputs did not arrive");
    } else {
        CK(cudaStreamSynchronize(h->stream));
    }
    std::memcpy(cmd, h->h_io + io_cmd(h->pb), sizeof(float) * d);
    if (info) {
        info->best_cost = st->best;
        info->mean_weighted_cost = st->wmean;
        info->status = st->status;
        info->step = st->step - 1;
    }
    return st->status;
}

int storm_step_async(storm_handle* h, const float* state_dev, const float* goal_dev, float* cmd_dev)
{
    if (!h || !state_dev || !goal_dev || !cmd_dev) return fail(h, STORM_ERR_INVALID_ARG, "NULL argument");
    const int d = h->pb.d;
    float* s_in = h->d_io + io_state(h->pb);
    float* g_in = h->d_io + io_goal(h->pb);
    float* c_out = h->d_io + io_cmd(h->pb);
    if (state_dev != s_in)
        CK(cudaMemcpyAsync(s_in, state_dev, sizeof(float) * 3 * d, cudaMemcpyDeviceToDevice, h->stream));
    if (goal_dev != g_in)
        CK(cudaMemcpyAsync(g_in, goal_dev, sizeof(float) * 7, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaGraphLaunch(h->g_dev, h->stream));
    if (cmd_dev != c_out)
        CK(cudaMemcpyAsync(cmd_dev, c_out, sizeof(float) * d, cudaMemcpyDeviceToDevice, h->stream));
    return STORM_OK;
}

int storm_sync(storm_handle* h, storm_step_info* info)
{
    if (!h) return STORM_ERR_INVALID_ARG;
    StepState st;
    CK(cudaMemcpyAsync(&st, h->d_st, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (info) {
        info->best_cost = st.best;
        info->mean_weighted_cost = st.wmean;
        info->status = st.status;
        info->step = st.step ? st.step - 1 : 0;
    }
    return st.status;
}

int storm_device_io(storm_handle* h, float** state_dev, float** goal_dev, float** cmd_dev)
{
    if (!h) return STORM_ERR_INVALID_ARG;
    if (state_dev) *state_dev = h->d_io + io_state(h->pb);
    if (goal_dev) *goal_dev = h->d_io + io_goal(h->pb);
    if (cmd_dev) *cmd_dev = h->d_io + io_cmd(h->pb);
    return STORM_OK;
}

int storm_shift(storm_handle* h)
{
    if (!h) return STORM_ERR_INVALID_ARG;
    const int O = h->pb.H * h->pb.d;
    k_shift<<<1, std::max(32, ((O + 3) / 4 + 31) / 32 * 32), 0, h->stream>>>(h->pb, h->d_st, 1);
    CK(cudaGetLastError());
    return STORM_OK;
}

int storm_sample_noise(storm_handle* h, uint32_t step, int iter, float* eps_dev)
{
    if (!h || !eps_dev) return fail(h, STORM_ERR_INVALID_ARG, "NULL argument");
    if (iter < 0 || iter > 255) return fail(h, STORM_ERR_INVALID_ARG, "bad iter");
    const uint32_t blocks = (static_cast<uint32_t>(h->pb.N) * h->pb.S * h->pb.d + 3) / 4;
    k_noise<<<(blocks + 255) / 256, 256, 0, h->stream>>>(h->pb, step, iter, eps_dev);
    CK(cudaGetLastError());
    return STORM_OK;
}

int storm_philox_words(storm_handle* h, uint32_t step, int iter, uint32_t first_block, int count,
                       uint32_t* words_dev)
{
    if (!h || !words_dev) return fail(h, STORM_ERR_INVALID_ARG, "NULL argument");
    if (iter < 0 || iter > 255 || count < 1 || count > (1 << 24))
        return fail(h, STORM_ERR_INVALID_ARG, "bad iter or count");
    if (reinterpret_cast<uintptr_t>(words_dev) % 16 != 0)
        return fail(h, STORM_ERR_INVALID_ARG, "words_dev must be 16-byte aligned");
    k_philox_words<<<(count + 255) / 256, 256, 0, h->stream>>>(h->pb, step, iter, first_block, count, words_dev);
    CK(cudaGetLastError());
    return STORM_OK;
}

int storm_generate_rollouts(storm_handle* h, const float* state_dev, const float* goal_dev,
                            uint32_t step, int iter, float* u_dev, float* theta_dev,
                            float* theta_dot_dev, float* ee_dev, float* terms_dev,
                            float* cost_dev, float* Ctot_dev)
{
    if (!h || !state_dev || !goal_dev) return fail(h, STORM_ERR_INVALID_ARG, "NULL argument");
    if (iter < 0 || iter > 255 || step > 0x7fffffffu) return fail(h, STORM_ERR_INVALID_ARG, "bad iter/step");
    RolloutOut out{u_dev ? u_dev : h->d_u, theta_dev, theta_dot_dev, ee_dev, terms_dev, cost_dev,
                   Ctot_dev ? Ctot_dev : h->d_C};
    return launch_rollout(h, h->stream, out, state_dev, goal_dev, static_cast<int>(step), iter);
}

int storm_cost_grad(storm_handle* h, const float* state_dev, const float* goal_dev,
                    const float* mean_dev, uint32_t step, int iter, float* grad_dev, float* J_dev,
                    float* Ctot_dev)
{
    if (!h || !state_dev || !goal_dev || !mean_dev || !grad_dev || !J_dev)
        return fail(h, STORM_ERR_INVALID_ARG, "NULL argument");
    if (iter < 0 || iter > 255 || step > 0x7fffffffu) return fail(h, STORM_ERR_INVALID_ARG, "bad iter/step");
    if (h->pb.filter != STORM_FILTER_DEFAULT || h->pb.w_ee_vel != 0.f || h->pb.w_ee_acc != 0.f ||
        h->pb.w_ball != 0.f)
        return fail(h, STORM_ERR_INVALID_ARG, "the adjoint needs the default filter and no ee / ball terms");
    return launch_adjoint(h, h->stream, state_dev, goal_dev, mean_dev, static_cast<int>(step), iter,
                          grad_dev, J_dev, Ctot_dev, 0.f, nullptr, 0);
}

int storm_update_distribution(storm_handle* h, const float* Ctot_dev, const float* u_dev,
                              float* weights_dev)
{
    if (!h || !Ctot_dev || !u_dev) return fail(h, STORM_ERR_INVALID_ARG, "NULL argument");
    return launch_update(h, h->stream, Ctot_dev, u_dev, weights_dev, nullptr, 0);
}

int storm_get_distribution(storm_handle* h, float* mean, float* sigma)
{
    if (!h) return STORM_ERR_INVALID_ARG;
    if (mean)
        CK(cudaMemcpyAsync(mean, h->pb.mu, sizeof(float) * h->pb.H * h->pb.d, cudaMemcpyDeviceToHost,
                           h->stream));
    if (sigma)
        CK(cudaMemcpyAsync(sigma, h->pb.sigma, sizeof(float) * h->pb.d, cudaMemcpyDeviceToHost,
                           h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return STORM_OK;
}

int storm_set_distribution(storm_handle* h, const float* mean, const float* sigma)
{
    if (!h) return STORM_ERR_INVALID_ARG;
    if (mean)
        CK(cudaMemcpyAsync(h->pb.mu, mean, sizeof(float) * h->pb.H * h->pb.d, cudaMemcpyHostToDevice,
                           h->stream));
    if (sigma)
        CK(cudaMemcpyAsync(h->pb.sigma, sigma, sizeof(float) * h->pb.d, cudaMemcpyHostToDevice,
                           h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return STORM_OK;
}

int storm_set_world(storm_handle* h, const storm_world* world)
{
    if (!h || !world) return fail(h, STORM_ERR_INVALID_ARG, "NULL argument");
    if (world->n_boxes < 0 || world->n_boxes > h->cap_boxes || world->n_spheres < 0 ||
        world->n_spheres > h->cap_wsph)
        return fail(h, STORM_ERR_INVALID_ARG, "obstacle count out of range");
    if ((world->n_boxes && !world->boxes) || (world->n_spheres && !world->spheres))
        return fail(h, STORM_ERR_INVALID_ARG, "NULL obstacle table");
    if (!finite_all(world->boxes, 6 * world->n_boxes) || !finite_all(world->spheres, 4 * world->n_spheres))
        return fail(h, STORM_ERR_INVALID_ARG, "non-finite obstacle");
    CK(cudaStreamSynchronize(h->stream));
    const int old_B = h->pb.B, old_O = h->pb.O;
    const int rc = upload_world(h, world);
    if (rc) return rc;
    // the counts are baked into the captured graphs and the shared-memory plan
    if (h->pb.B != old_B || h->pb.O != old_O) {
        const RolloutLayout L = rollout_layout(h->pb);
        h->rollout_smem = L.bytes;
        return build_graphs(h);
    }
    return STORM_OK;
}

int storm_forward_kinematics(storm_handle* h, const float* theta_dev, int count, float* ee_dev)
{
    if (!h || count < 0 || (count > 0 && (!theta_dev || !ee_dev)))
        return fail(h, STORM_ERR_INVALID_ARG, "bad argument");
    if (count == 0) return STORM_OK;
    k_fk<<<(count + 127) / 128, 128, 0, h->stream>>>(h->pb, theta_dev, count, ee_dev);
    CK(cudaGetLastError());
    return STORM_OK;
}

int storm_ee_twist(storm_handle* h, const float* theta_dev, const float* theta_dot_dev,
                   const float* theta_ddot_dev, int count, float* xd_dev, float* xdd_dev)
{
    if (!h || count < 0 ||
        (count > 0 && (!theta_dev || !theta_dot_dev || !theta_ddot_dev || !xd_dev || !xdd_dev)))
        return fail(h, STORM_ERR_INVALID_ARG, "bad argument");
    if (count == 0) return STORM_OK;
    k_ee_twist<<<(count + 127) / 128, 128, 0, h->stream>>>(h->pb, theta_dev, theta_dot_dev, theta_ddot_dev, count,
                                                          xd_dev, xdd_dev);
    CK(cudaGetLastError());
    return STORM_OK;
}

int storm_set_ball(storm_handle* h, const float* ball)
{
    if (!h || !ball) return fail(h, STORM_ERR_INVALID_ARG, "NULL argument");
    for (int i = 0; i < 6; ++i)
        if (!std::isfinite(ball[i])) return fail(h, STORM_ERR_INVALID_ARG, "non-finite ball state");
    std::memcpy(h->h_ball, ball, sizeof(float) * 6);
    CK(cudaMemcpyAsync(h->d_ball, h->h_ball, sizeof(float) * 6, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return STORM_OK;
}

int storm_set_trace(storm_handle* h, unsigned long long* trace_dev)
{
    if (!h) return STORM_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->stream));
    h->pb.trace = trace_dev;
    return build_graphs(h);
}

int storm_set_broadphase(storm_handle* h, int on)
{
    if (!h) return STORM_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->stream));
    h->pb.broadphase = on ? 1 : 0;
    return build_graphs(h);
}

int storm_get_launch(const storm_handle* h, int* ppc, int* threads)
{
    if (!h) return STORM_ERR_INVALID_ARG;
    if (h->mapping != STORM_MAP_CTA) {
        if (ppc) *ppc = h->wpc * warp_plan(h->pb, 1).PW;
        if (threads) *threads = h->wpc * 32 * warps_per_group(h->mapping);
    } else {
        if (ppc) *ppc = h->pb.ppc;
        if (threads) *threads = h->threads;
    }
    return STORM_OK;
}

int storm_get_launch_mapping(const storm_handle* h) { return h ? h->mapping : STORM_ERR_INVALID_ARG; }

int storm_set_dependent_launch(storm_handle* h, int on)
{
    if (!h || (on != 0 && on != 1)) return STORM_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->stream));
    h->dep_launch = on == 1;
    return build_graphs(h);
}

int storm_get_dependent_launch(const storm_handle* h) { return h ? (h->dep_launch ? 1 : 0) : STORM_ERR_INVALID_ARG; }

static int set_launch_warp_impl(storm_handle* h, int wpc, bool rebuild, int mapping = STORM_MAP_WARP)
{
    const int kw = warps_per_group(mapping);
    if (wpc < 1 || wpc > kWarpMaxWarps / kw) return fail(h, STORM_ERR_INVALID_ARG, "warps per CTA out of range");
    const WarpPlan wp = warp_plan(h->pb, kw);
    const size_t bytes = sizeof(float) * size_t(wp.floats) * wpc;
    int optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    if (bytes > size_t(optin)) return fail(h, STORM_ERR_INVALID_ARG, "launch shape needs too much shared memory");
    h->mapping = mapping;
    h->wpc = wpc;
    h->warp_smem = bytes;
    h->warp_grid = (h->pb.N + wp.PW * wpc - 1) / (wp.PW * wpc);
    return rebuild ? build_graphs(h) : STORM_OK;
}

int storm_set_launch_warp(storm_handle* h, int warps_per_cta)
{
    if (!h) return STORM_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->stream));
    return set_launch_warp_impl(h, warps_per_cta, true);
}

int storm_set_launch_warp_pair(storm_handle* h, int pairs_per_cta)
{
    if (!h) return STORM_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->stream));
    return set_launch_warp_impl(h, pairs_per_cta, true, STORM_MAP_WARP_PAIR);
}

int storm_set_launch_warp_quad(storm_handle* h, int groups_per_cta)
{
    if (!h) return STORM_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->stream));
    return set_launch_warp_impl(h, groups_per_cta, true, STORM_MAP_WARP_QUAD);
}

static int set_launch_impl(storm_handle* h, int ppc, int threads, bool rebuild)
{
    if (ppc < 1 || ppc > h->pb.N || threads < 64 || threads > kMaxThreads || threads % 32)
        return fail(h, STORM_ERR_INVALID_ARG, "launch shape out of range");
    Problem trial = h->pb;
    trial.ppc = ppc;
    const RolloutLayout L = rollout_layout(trial);
    int optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    if (L.bytes > optin) return fail(h, STORM_ERR_INVALID_ARG, "launch shape needs too much shared memory");
    h->pb.ppc = ppc;
    h->threads = threads;
    h->grid = (h->pb.N + ppc - 1) / ppc;
    h->rollout_smem = L.bytes;
    h->mapping = STORM_MAP_CTA;
    return rebuild ? build_graphs(h) : STORM_OK;
}

int storm_set_launch(storm_handle* h, int ppc, int threads)
{
    if (!h) return STORM_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->stream));
    return set_launch_impl(h, ppc, threads, true);
}

int storm_autotune(storm_handle* h, float* best_us)
{
    if (!h) return STORM_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->stream));
    const int ppcs[] = {1, 2, 3, 4, 6, 8, 12, 16};
    const int ths[] = {128, 256, 512};
    const int wpcs[] = {1, 2, 4, 8};
    const int pairs[] = {1, 2, 4};
    const int quads[] = {1, 2};
    const int old_map = h->mapping, old_ppc = h->pb.ppc, old_threads = h->threads, old_wpc = h->wpc;
    float best = INFINITY;
    int best_map = old_map, best_ppc = old_ppc, best_threads = old_threads, best_wpc = old_wpc;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    RolloutOut out{h->d_u, nullptr, nullptr, nullptr, nullptr, nullptr, h->d_C};
    const float* state = h->d_io + io_state(h->pb);
    const float* goal = h->d_io + io_goal(h->pb);
    int rc = STORM_OK;
    auto measure = [&]() {  // median of 10 timed launches after 3 warm-up launches
        std::vector<float> t;
        for (int it = 0; it < 13 && rc == STORM_OK; ++it) {
            cudaEventRecord(e0, h->stream);
            rc = launch_rollout(h, h->stream, out, state, goal, 0, 0);
            cudaEventRecord(e1, h->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = STORM_ERR_CUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (it >= 3) t.push_back(ms * 1e3f);
        }
        if (rc) return INFINITY;
        std::sort(t.begin(), t.end());
        return t[t.size() / 2];
    };
    for (int ppc : ppcs) {
        if (ppc > h->pb.N || ppc * h->pb.H > kMaxThreads) continue;
        for (int th : ths) {
            if (set_launch_impl(h, ppc, th, false) != STORM_OK) continue;
            const float med = measure();
            if (rc) break;
            if (med < best) {
                best = med;
                best_map = STORM_MAP_CTA;
                best_ppc = ppc;
                best_threads = th;
            }
        }
        if (rc) break;
    }
    for (int w : wpcs) {
        if (rc) break;
        if (set_launch_warp_impl(h, w, false) != STORM_OK) continue;
        const float med = measure();
        if (rc) break;
        if (med < best) {
            best = med;
            best_map = STORM_MAP_WARP;
            best_wpc = w;
        }
    }
    // More pairs per CTA means fewer CTAs: at 500 particles four pairs a CTA leave
    // 23 of the 148 SMs idle, and the control step ran ~3 % slower than with one
    // pair a CTA although single rollouts timed here were within noise of each
    // other (two pairs a CTA, 250 CTAs, ran the step 0.5 % faster than one).
    // So a pair shape whose grid leaves SMs idle is taken only if it beats the
    // best so far by 5 %.
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) rc = STORM_ERR_CUDA;
    float best_pair = INFINITY;
    int best_pair_wpc = 1;
    for (int w : pairs) {
        if (rc) break;
        if (set_launch_warp_impl(h, w, false, STORM_MAP_WARP_PAIR) != STORM_OK) continue;
        const bool fills = h->warp_grid >= sms;
        const float med = measure();
        if (rc) break;
        if (med < (fills ? 1.f : 0.95f) * best_pair) {
            best_pair = med;
            best_pair_wpc = w;
        }
    }
    if (best_pair < best) {
        best = best_pair;
        best_map = STORM_MAP_WARP_PAIR;
        best_wpc = best_pair_wpc;
    }
    for (int w : quads) {
        if (rc) break;
        if (set_launch_warp_impl(h, w, false, STORM_MAP_WARP_QUAD) != STORM_OK) continue;
        const float med = measure();
        if (rc) break;
        if (med < best) {
            best = med;
            best_map = STORM_MAP_WARP_QUAD;
            best_wpc = w;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // The tuning state is one state: where the arm folds or meets obstacles the
    // collision work per item grows several times, and the pair mapping shares
    // it between its two warps while the others do not.  So the pair mapping is
    // kept unless another shape beats it by more than 5 % here.
    if (best_map != STORM_MAP_WARP_PAIR && best_pair <= 1.05f * best) {
        best = best_pair;
        best_map = STORM_MAP_WARP_PAIR;
        best_wpc = best_pair_wpc;
    }
    h->err = "no error";  // shapes that did not fit are not errors of the handle
    if (rc) {
        if (old_map != STORM_MAP_CTA) {
            set_launch_impl(h, old_ppc, old_threads, false);
            set_launch_warp_impl(h, old_wpc, true, old_map);
        } else {
            set_launch_warp_impl(h, old_wpc, false);
            set_launch_impl(h, old_ppc, old_threads, true);
        }
        return rc;
    }
    if (best_us) *best_us = best;
    if (best_map != STORM_MAP_CTA) {
        set_launch_impl(h, best_ppc, best_threads, false);  // keep the CTA-mapping shape consistent
        return set_launch_warp_impl(h, best_wpc, true, best_map);
    }
    set_launch_warp_impl(h, best_wpc, false);
    return set_launch_impl(h, best_ppc, best_threads, true);
}

// checkpoint blob: magic, version, N, H, d, step | mu (H*d) | sigma (d)
static const uint32_t kMagic = 0x4d525453u;  // "STRM"

int storm_get_state(storm_handle* h, void* buf, size_t* len)
{
    if (!h || !len) return STORM_ERR_INVALID_ARG;
    const int O = h->pb.H * h->pb.d;
    const size_t need = 6 * 4 + 4 * (O + h->pb.d);
    if (!buf) {
        *len = need;
        return STORM_OK;
    }
    if (*len < need) return fail(h, STORM_ERR_INVALID_ARG, "buffer too small");
    StepState st;
    uint32_t* w = static_cast<uint32_t*>(buf);
    CK(cudaMemcpyAsync(&st, h->d_st, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(w + 6, h->pb.mu, 4 * O, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(w + 6 + O, h->pb.sigma, 4 * h->pb.d, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    w[0] = kMagic;
    w[1] = 1;
    w[2] = h->pb.N;
    w[3] = h->pb.H;
    w[4] = h->pb.d;
    w[5] = st.step;
    *len = need;
    return STORM_OK;
}

int storm_set_state(storm_handle* h, const void* buf, size_t len)
{
    if (!h || !buf) return STORM_ERR_INVALID_ARG;
    const int O = h->pb.H * h->pb.d;
    const size_t need = 6 * 4 + 4 * (O + h->pb.d);
    const uint32_t* w = static_cast<const uint32_t*>(buf);
    if (len != need || w[0] != kMagic || w[1] != 1 || w[2] != uint32_t(h->pb.N) ||
        w[3] != uint32_t(h->pb.H) || w[4] != uint32_t(h->pb.d))
        return fail(h, STORM_ERR_STATE, "checkpoint does not match this handle");
    StepState st{w[5], 0, 0.f, 0.f};
    CK(cudaMemcpyAsync(h->pb.mu, w + 6, 4 * O, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->pb.sigma, w + 6 + O, 4 * h->pb.d, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->d_st, &st, sizeof(st), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return STORM_OK;
}

}  // extern "C"

// ============================================================================ FP32 peak
//
// The FP32 FMA rate of this GPU, measured: every thread runs eight independent
// chains of fused multiply-adds on registers (no memory traffic), either one
// FMA per instruction or Blackwell's paired FMA (two per instruction), with the
// whole GPU occupied.  The ALU roofline of the rollout kernel divides by it.
template <bool kPaired>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, float seed, float* __restrict__ sink)
{
    const float m = 0.9999f, c = 1e-7f;
    float acc = 0.f;
    if (kPaired) {
        float2 a[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = make_float2(seed + threadIdx.x + k, seed - k);
        const float2 m2 = make_float2(m, m), c2 = make_float2(c, -c);
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = __ffma2_rn(a[k], m2, c2);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc += a[k].x + a[k].y;
    } else {
        float a[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) a[k] = seed + threadIdx.x + k;
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < 16; ++k) a[k] = fmaf(a[k], m, c);
#pragma unroll
        for (int k = 0; k < 16; ++k) acc += a[k];
    }
    if (acc == seed) sink[blockIdx.x] = acc;  // keeps the chains live; never true in practice
}

extern "C" int storm_fp32_peak(int iters, float* tflops_scalar, float* tflops_paired)
{
    if (iters < 1 || iters > (1 << 24) || !tflops_scalar || !tflops_paired) return STORM_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return STORM_ERR_CUDA;
    }
    const int blocks = sms * 8;  // 2048 threads per SM
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float* sink = nullptr;
    int rc = STORM_OK;
    auto ck = [&](cudaError_t e) {
        if (rc == STORM_OK && e != cudaSuccess) {
            (void)cudaGetLastError();
            rc = STORM_ERR_CUDA;
        }
    };
    ck(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    ck(cudaEventCreate(&e0));
    ck(cudaEventCreate(&e1));
    ck(cudaMalloc(&sink, sizeof(float) * blocks));
    const double flops = 2.0 * 16.0 * iters * blocks * 256.0;  // 16 FMAs per iteration per thread
    for (int paired = 0; paired < 2 && rc == STORM_OK; ++paired) {
        auto launch = [&]() {
            if (paired)
                k_fma_peak<true><<<blocks, 256, 0, s>>>(iters, 1.0f, sink);
            else
                k_fma_peak<false><<<blocks, 256, 0, s>>>(iters, 1.0f, sink);
        };
        launch();  // warm-up
        ck(cudaGetLastError());
        float best = 0.f;
        for (int r = 0; r < 5 && rc == STORM_OK; ++r) {
            ck(cudaEventRecord(e0, s));
            launch();
            ck(cudaEventRecord(e1, s));
            ck(cudaEventSynchronize(e1));
            float ms = 0.f;
            ck(cudaEventElapsedTime(&ms, e0, e1));
            if (rc == STORM_OK && ms > 0.f) best = std::max(best, static_cast<float>(flops / (ms * 1e-3) / 1e12));
        }
        (paired ? *tflops_paired : *tflops_scalar) = best;
    }
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    return rc;
}

// ============================================================================ no allocation
//
// storm_rollout_costs_noalloc: the rollout kernel launched on tables and a
// control batch that live in this file-scope static array instead of memory
// from cudaMalloc.  Host code must not use the array's name as a device
// address; the per-device address comes from cudaGetSymbolAddress.

static __device__ __align__(256) unsigned char g_noalloc_scratch[STORM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoallocMaxDevices] = {};

// Once per device, with that device current: the scratch address and the
// rollout kernel's shared-memory opt-in.
int noalloc_setup(int dev, void** addr, std::string& msg)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            msg = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return STORM_ERR_CUDA;
        }
        int optin = 0;
        cudaFuncAttributes ra;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&ra, k_rollout);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_rollout, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - static_cast<int>(ra.sharedSizeBytes));
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            msg = std::string("rollout kernel attribute: ") + cudaGetErrorString(e);
            return STORM_ERR_CUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *addr = g_noalloc_addr[dev];
    return STORM_OK;
}

}  // namespace

extern "C" int storm_rollout_costs_noalloc(const storm_robot* r, const storm_world* w,
                                           const storm_params* p, const float* state_dev,
                                           const float* goal_dev, const float* mean_dev,
                                           const float* sigma_dev, uint32_t step, int iter,
                                           float* Ctot_dev, void* cuda_stream)
{
    std::string msg;
    const int v = validate(r, w, p, msg);
    if (v) return v;
    if (!state_dev || !goal_dev || !mean_dev || !sigma_dev || !Ctot_dev) return STORM_ERR_INVALID_ARG;
    if (iter < 0 || iter > 255 || step > 0x7fffffffu) return STORM_ERR_INVALID_ARG;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    {
        // the table copies below read pageable host vectors that die with this
        // call: a captured graph would replay copies from freed memory
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            (void)cudaGetLastError();
            fprintf(stderr, "storm_rollout_costs_noalloc: the stream is being captured (not supported)\n");
            return STORM_ERR_INVALID_ARG;
        }
    }

    // the problem and its host tables exactly as storm_create builds them
    // (spheres sorted by link, link-pair blocks, link bounds, broad phase on)
    Problem pb{};
    HostTables ht;
    fill_problem(r, w, p, pb, ht);

    // scratch plan: the model tables (with the Halton noise when that sampler
    // is chosen), then the N x H x d control batch
    const TablePlan t = plan_tables(pb, std::max(pb.B, 1), std::max(pb.O, 1), static_cast<int>(ht.raw.size()));
    const size_t u_off = (t.total + 255) & ~size_t(255);
    const size_t u_bytes = sizeof(float) * size_t(pb.N) * pb.H * pb.d;
    if (u_off + u_bytes > STORM_NOALLOC_SCRATCH_BYTES) {
        fprintf(stderr,
                "storm_rollout_costs_noalloc: problem needs %zu bytes of scratch, more than the "
                "%u-byte static scratch\n",
                u_off + u_bytes, STORM_NOALLOC_SCRATCH_BYTES);
        return STORM_ERR_INVALID_ARG;
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
        (void)cudaGetLastError();
        return STORM_ERR_CUDA;
    }
    void* addr = nullptr;
    int rc = noalloc_setup(dev, &addr, msg);
    if (rc) {
        fprintf(stderr, "storm_rollout_costs_noalloc: %s\n", msg.c_str());
        return rc;
    }
    char* base = static_cast<char*>(addr);
    float* d_u = reinterpret_cast<float*>(base + u_off);
    // every table the rollout reads is rewritten here (host copies, then the
    // set-up kernels), so nothing an earlier call left in the scratch is used
    cudaError_t e = upload_problem(pb, ht, base, t, stream);
    if (e == cudaSuccess) {
        pb.mu = const_cast<float*>(mean_dev);  // read only by the rollout kernel
        pb.sigma = const_cast<float*>(sigma_dev);
        const RolloutLayout L = rollout_layout(pb);
        RolloutOut out{d_u, nullptr, nullptr, nullptr, nullptr, nullptr, Ctot_dev};
        const int grid = (pb.N + pb.ppc - 1) / pb.ppc;
        k_rollout<<<grid, kThreads, L.bytes, stream>>>(pb, out, state_dev, goal_dev, nullptr,
                                                      static_cast<int>(step), iter);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        fprintf(stderr, "storm_rollout_costs_noalloc: %s\n", cudaGetErrorString(e));
        return STORM_ERR_CUDA;
    }
    return STORM_OK;
}

// ============================================================================ batch host runtime

struct storm_batch {
    int device = 0;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    bool own_stream = false;
    int n = 0, Kmax = 1;
    int threads = kThreads, items = 64;
    int mapping = STORM_MAP_WARP;  // rollout work mapping (CTA tiles or warp tasks)
    bool full = false;             // an instance needs the full warp rollout (see rollout_warp_body)
    int wpc = 4;                   // warps per CTA of the warp mapping
    std::vector<BatchInstance> inst;  // host mirror of d_inst
    std::vector<int> dof, state_off, cmd_off;
    std::vector<double> sigma_init;
    int state_floats = 0, cmd_floats = 0;
    void* arena = nullptr;
    BatchInstance* d_inst = nullptr;
    BatchTile* d_tiles = nullptr;
    int2* d_tasks = nullptr;  // (instance, particle group) of the warp mapping
    int n_tasks = 0, warp_floats = 0;
    int n_tiles = 0, grid = 0;
    float* d_in = nullptr;   // states | goals
    float* d_out = nullptr;  // cmds | StepState x n
    float* h_in = nullptr;
    float* h_out = nullptr;
    size_t rollout_smem = 0, update_smem = 0;
    cudaGraphExec_t g_host = nullptr, g_dev = nullptr;
    std::string err = "no error";
};

namespace {

#define BK(call)                                                                  \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            (void)cudaGetLastError();                                             \
            b->err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
            return e_ == cudaErrorMemoryAllocation ? STORM_ERR_OOM : STORM_ERR_CUDA; \
        }                                                                         \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t out_st_offset(const storm_batch* b) { return align256(sizeof(float) * b->cmd_floats); }

// Tiles of `items` (particle, step) work items per CTA, largest first.
int batch_tiles(storm_batch* b, int items, std::vector<BatchTile>& tiles, size_t& smem)
{
    tiles.clear();
    smem = 0;
    std::vector<std::pair<double, BatchTile>> w;
    for (int i = 0; i < b->n; ++i) {
        Problem pb = b->inst[i].pb;
        pb.ppc = std::max(1, std::min(pb.N, items / pb.H));
        b->inst[i].pb.ppc = pb.ppc;
        smem = std::max(smem, static_cast<size_t>(rollout_layout(pb).bytes));
        const double per_item = 100.0 + pb.M * (pb.B + pb.O) + 49.0 * pb.NPB + pb.P;
        for (int n0 = 0; n0 < pb.N; n0 += pb.ppc) {
            const int np = std::min(pb.ppc, pb.N - n0);
            w.push_back({np * pb.H * per_item, BatchTile{i, n0, np, 0}});
        }
    }
    std::stable_sort(w.begin(), w.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    for (auto& e : w) tiles.push_back(e.second);
    return STORM_OK;
}

int batch_apply_launch(storm_batch* b, int items, int threads)
{
    std::vector<BatchTile> tiles;
    size_t smem = 0;
    batch_tiles(b, items, tiles, smem);
    int optin = 0, sms = 0;
    BK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
    BK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    cudaFuncAttributes fa;
    BK(cudaFuncGetAttributes(&fa, k_rollout_batch));
    if (smem + fa.sharedSizeBytes > size_t(optin)) {
        b->err = "tile shape needs too much shared memory";
        return STORM_ERR_INVALID_ARG;
    }
    BK(cudaFuncSetAttribute(k_rollout_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            optin - static_cast<int>(fa.sharedSizeBytes)));
    int per_sm = 0;
    BK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rollout_batch, threads, smem));
    if (per_sm < 1) {
        b->err = "tile shape does not fit an SM";
        return STORM_ERR_INVALID_ARG;
    }
    if (b->d_tiles) cudaFree(b->d_tiles);
    b->d_tiles = nullptr;
    BK(cudaMalloc(&b->d_tiles, sizeof(BatchTile) * tiles.size()));
    BK(cudaMemcpyAsync(b->d_tiles, tiles.data(), sizeof(BatchTile) * tiles.size(),
                       cudaMemcpyHostToDevice, b->stream));
    BK(cudaMemcpyAsync(b->d_inst, b->inst.data(), sizeof(BatchInstance) * b->n,
                       cudaMemcpyHostToDevice, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    b->n_tiles = static_cast<int>(tiles.size());
    b->grid = std::min(b->n_tiles, per_sm * sms);
    b->rollout_smem = smem;
    b->items = items;
    b->threads = threads;
    b->mapping = STORM_MAP_CTA;
    return STORM_OK;
}

// Warp mapping: one task per (instance, group of PW particles), largest first;
// every warp's shared region is sized for the largest instance.
int batch_apply_launch_warp(storm_batch* b, int wpc)
{
    if (wpc < 1 || wpc > kWarpMaxWarps) {
        b->err = "warps per CTA must be in 1..8";
        return STORM_ERR_INVALID_ARG;
    }
    std::vector<std::pair<double, int2>> w;
    int floats = 0;
    for (int i = 0; i < b->n; ++i) {
        const Problem& pb = b->inst[i].pb;
        const WarpPlan wp = warp_plan(pb, 1);
        floats = std::max(floats, wp.floats);
        const double per_item = 100.0 + pb.M * (pb.B + pb.O) + 49.0 * pb.NPB + pb.P;
        for (int g = 0; g * wp.PW < pb.N; ++g)
            w.push_back({std::min(wp.PW, pb.N - g * wp.PW) * pb.H * per_item, make_int2(i, g)});
    }
    std::stable_sort(w.begin(), w.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    std::vector<int2> tasks;
    for (auto& e : w) tasks.push_back(e.second);
    const size_t smem = sizeof(float) * size_t(floats) * wpc;
    int optin = 0, sms = 0;
    BK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
    BK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    const auto kernel = b->full ? k_rollout_warp_batch<true> : k_rollout_warp_batch<false>;
    cudaFuncAttributes fa;
    BK(cudaFuncGetAttributes(&fa, kernel));
    if (smem + fa.sharedSizeBytes > size_t(optin)) {
        b->err = "warp shape needs too much shared memory";
        return STORM_ERR_INVALID_ARG;
    }
    BK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            optin - static_cast<int>(fa.sharedSizeBytes)));
    int per_sm = 0;
    BK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, wpc * 32, smem));
    if (per_sm < 1) {
        b->err = "warp shape does not fit an SM";
        return STORM_ERR_INVALID_ARG;
    }
    if (b->d_tasks) cudaFree(b->d_tasks);
    b->d_tasks = nullptr;
    BK(cudaMalloc(&b->d_tasks, sizeof(int2) * tasks.size()));
    BK(cudaMemcpyAsync(b->d_tasks, tasks.data(), sizeof(int2) * tasks.size(), cudaMemcpyHostToDevice,
                       b->stream));
    BK(cudaMemcpyAsync(b->d_inst, b->inst.data(), sizeof(BatchInstance) * b->n,
                       cudaMemcpyHostToDevice, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    b->n_tasks = static_cast<int>(tasks.size());
    b->grid = std::min((b->n_tasks + wpc - 1) / wpc, per_sm * sms);
    b->rollout_smem = smem;
    b->warp_floats = floats;
    b->wpc = wpc;
    b->mapping = STORM_MAP_WARP;
    return STORM_OK;
}

cudaError_t batch_launch_rollout(storm_batch* b, cudaStream_t s, int iter)
{
    if (b->mapping == STORM_MAP_WARP && b->full)
        k_rollout_warp_batch<true><<<b->grid, b->wpc * 32, b->rollout_smem, s>>>(b->d_inst, b->d_tasks, b->n_tasks,
                                                                                 iter, b->warp_floats);
    else if (b->mapping == STORM_MAP_WARP)
        k_rollout_warp_batch<false><<<b->grid, b->wpc * 32, b->rollout_smem, s>>>(b->d_inst, b->d_tasks,
                                                                                  b->n_tasks, iter, b->warp_floats);
    else
        k_rollout_batch<<<b->grid, b->threads, b->rollout_smem, s>>>(b->d_inst, b->d_tiles, b->n_tiles, iter);
    return cudaGetLastError();
}

int batch_enqueue(storm_batch* b, cudaStream_t s)
{
    k_shift_batch<<<b->n, 128, 0, s>>>(b->d_inst);
    BK(cudaGetLastError());
    for (int k = 0; k < b->Kmax; ++k) {
        BK(batch_launch_rollout(b, s, k));
        k_update_batch<<<b->n * kUpdCluster, kUpdateThreads, b->update_smem, s>>>(b->d_inst, k);
        BK(cudaGetLastError());
    }
    return STORM_OK;
}

void batch_destroy_graphs(storm_batch* b)
{
    if (b->g_dev) cudaGraphExecDestroy(b->g_dev);
    if (b->g_host) cudaGraphExecDestroy(b->g_host);
    b->g_dev = b->g_host = nullptr;
}

int batch_build_graphs(storm_batch* b)
{
    batch_destroy_graphs(b);
    for (int with_io = 0; with_io < 2; ++with_io) {
        cudaGraph_t g = nullptr;
        BK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = STORM_OK;
        const size_t in_bytes = sizeof(float) * (b->state_floats + 7 * b->n);
        const size_t out_bytes = out_st_offset(b) + sizeof(StepState) * b->n;
        if (with_io && cudaMemcpyAsync(b->d_in, b->h_in, in_bytes, cudaMemcpyHostToDevice, b->cap_stream))
            rc = STORM_ERR_CUDA;
        if (!rc) rc = batch_enqueue(b, b->cap_stream);
        if (!rc && with_io &&
            cudaMemcpyAsync(b->h_out, b->d_out, out_bytes, cudaMemcpyDeviceToHost, b->cap_stream))
            rc = STORM_ERR_CUDA;
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        BK(e);
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        BK(e);
        (with_io ? b->g_host : b->g_dev) = ex;
    }
    return STORM_OK;
}

void batch_free(storm_batch* b)
{
    batch_destroy_graphs(b);
    if (b->arena) cudaFree(b->arena);
    if (b->d_inst) cudaFree(b->d_inst);
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_tasks) cudaFree(b->d_tasks);
    if (b->d_in) cudaFree(b->d_in);
    if (b->d_out) cudaFree(b->d_out);
    if (b->h_in) cudaFreeHost(b->h_in);
    if (b->h_out) cudaFreeHost(b->h_out);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

int batch_create_impl(storm_batch* b, int n, const storm_robot* r, const storm_world* w,
                      const storm_params* p, void* stream)
{
    BK(cudaGetDevice(&b->device));
    if (stream) {
        b->stream = static_cast<cudaStream_t>(stream);
    } else {
        BK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        b->own_stream = true;
    }
    BK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    b->n = n;
    b->inst.resize(n);
    std::vector<HostTables> ht(n);
    std::vector<TablePlan> plans(n);
    std::vector<size_t> off(n);
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
        BatchInstance& I = b->inst[i];
        I = BatchInstance{};
        fill_problem(r + i, w + i, p + i, I.pb, ht[i]);
        b->full = b->full || needs_full_rollout(I.pb);
        I.K = p[i].K;
        b->Kmax = std::max(b->Kmax, I.K);
        b->dof.push_back(r[i].dof);
        b->sigma_init.push_back(p[i].sigma_init);
        b->state_off.push_back(b->state_floats);
        b->cmd_off.push_back(b->cmd_floats);
        b->state_floats += 3 * r[i].dof;
        b->cmd_floats += r[i].dof;
        plans[i] = plan_tables(I.pb, std::max(I.pb.B, 1), std::max(I.pb.O, 1),
                               static_cast<int>(ht[i].raw.size()));
        off[i] = total;
        const Problem& pb = I.pb;
        total += align256(plans[i].total) + align256(sizeof(float) * size_t(pb.N) * pb.H * pb.d) +
                 align256(sizeof(float) * pb.N);
        b->update_smem = std::max(b->update_smem, sizeof(float) * 2 * ((pb.N + 3) & ~size_t(3)));
    }
    BK(cudaMalloc(&b->arena, total));
    BK(cudaMemsetAsync(b->arena, 0, total, b->stream));
    const size_t out_bytes = out_st_offset(b) + sizeof(StepState) * n;
    BK(cudaMalloc(&b->d_in, sizeof(float) * (b->state_floats + 7 * n)));
    BK(cudaMalloc(&b->d_out, out_bytes));
    BK(cudaMallocHost(&b->h_in, sizeof(float) * (b->state_floats + 7 * n)));
    BK(cudaMallocHost(&b->h_out, out_bytes));
    BK(cudaMemsetAsync(b->d_in, 0, sizeof(float) * (b->state_floats + 7 * n), b->stream));
    BK(cudaMemsetAsync(b->d_out, 0, out_bytes, b->stream));
    StepState* st = reinterpret_cast<StepState*>(reinterpret_cast<char*>(b->d_out) + out_st_offset(b));
    for (int i = 0; i < n; ++i) {
        BatchInstance& I = b->inst[i];
        char* base = static_cast<char*>(b->arena) + off[i];
        BK(upload_problem(I.pb, ht[i], base, plans[i], b->stream));
        char* q = base + align256(plans[i].total);
        I.u = reinterpret_cast<float*>(q);
        q += align256(sizeof(float) * size_t(I.pb.N) * I.pb.H * I.pb.d);
        I.C = reinterpret_cast<float*>(q);
        I.state = b->d_in + b->state_off[i];
        I.goal = b->d_in + b->state_floats + 7 * i;
        I.cmd = b->d_out + b->cmd_off[i];
        I.st = st + i;
        std::vector<float> sg(I.pb.d, static_cast<float>(p[i].sigma_init));
        BK(cudaMemcpyAsync(I.pb.sigma, sg.data(), 4 * I.pb.d, cudaMemcpyHostToDevice, b->stream));
    }
    BK(cudaMalloc(&b->d_inst, sizeof(BatchInstance) * n));
    int optin = 0;
    BK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
    cudaFuncAttributes ua;
    BK(cudaFuncGetAttributes(&ua, k_update_batch));
    if (b->update_smem + ua.sharedSizeBytes > size_t(optin)) {
        b->err = "update needs too much shared memory";
        return STORM_ERR_INVALID_ARG;
    }
    BK(cudaFuncSetAttribute(k_update_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            optin - static_cast<int>(ua.sharedSizeBytes)));
    const int rc = batch_apply_launch_warp(b, 4);
    if (rc) return rc;
    return batch_build_graphs(b);
}

}  // namespace

extern "C" {

const char* storm_batch_last_error(const storm_batch* b) { return b ? b->err.c_str() : "NULL batch"; }

int storm_batch_create(int count, const storm_robot* robots, const storm_world* worlds,
                       const storm_params* params, void* cuda_stream, storm_batch** out)
{
    if (!out) return STORM_ERR_INVALID_ARG;
    *out = nullptr;
    if (count < 1 || count > STORM_MAX_BATCH || !robots || !worlds || !params)
        return STORM_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        std::string msg;
        int v = validate(robots + i, worlds + i, params + i, msg);
        if (!v && params[i].w_ball != 0.0) {
            msg = "batched instances take no ball term (w_ball = 0)";
            v = STORM_ERR_INVALID_ARG;
        }
        if (v) {
            fprintf(stderr, "storm_batch_create: instance %d: %s\n", i, msg.c_str());
            return v;
        }
    }
    storm_batch* b = new (std::nothrow) storm_batch();
    if (!b) return STORM_ERR_OOM;
    const int rc = batch_create_impl(b, count, robots, worlds, params, cuda_stream);
    if (rc) {
        fprintf(stderr, "storm_batch_create: %s\n", b->err.c_str());
        batch_free(b);
        delete b;
        return rc;
    }
    *out = b;
    return STORM_OK;
}

void storm_batch_destroy(storm_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
    delete b;
}

int storm_batch_sizes(const storm_batch* b, int* state_floats, int* cmd_floats)
{
    if (!b) return STORM_ERR_INVALID_ARG;
    if (state_floats) *state_floats = b->state_floats;
    if (cmd_floats) *cmd_floats = b->cmd_floats;
    return STORM_OK;
}

int storm_batch_step(storm_batch* b, const float* states, const float* goals, float* cmds,
                     int* statuses)
{
    if (!b || !states || !goals || !cmds) return STORM_ERR_INVALID_ARG;
    for (int i = 0; i < b->state_floats; ++i)
        if (!std::isfinite(states[i])) return b->err = "non-finite state", STORM_ERR_NONFINITE;
    for (int i = 0; i < 7 * b->n; ++i)
        if (!std::isfinite(goals[i])) return b->err = "non-finite goal", STORM_ERR_NONFINITE;
    std::memcpy(b->h_in, states, sizeof(float) * b->state_floats);
    std::memcpy(b->h_in + b->state_floats, goals, sizeof(float) * 7 * b->n);
    BK(cudaGraphLaunch(b->g_host, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    std::memcpy(cmds, b->h_out, sizeof(float) * b->cmd_floats);
    const StepState* st =
        reinterpret_cast<const StepState*>(reinterpret_cast<const char*>(b->h_out) + out_st_offset(b));
    int worst = STORM_OK;
    for (int i = 0; i < b->n; ++i) {
        if (statuses) statuses[i] = st[i].status;
        worst = std::max(worst, st[i].status);
    }
    return worst;
}

int storm_batch_step_resident(storm_batch* b)
{
    if (!b) return STORM_ERR_INVALID_ARG;
    BK(cudaGraphLaunch(b->g_dev, b->stream));
    return STORM_OK;
}

int storm_batch_device_io(storm_batch* b, float** states_dev, float** goals_dev, float** cmds_dev)
{
    if (!b) return STORM_ERR_INVALID_ARG;
    if (states_dev) *states_dev = b->d_in;
    if (goals_dev) *goals_dev = b->d_in + b->state_floats;
    if (cmds_dev) *cmds_dev = b->d_out;
    return STORM_OK;
}

int storm_batch_sync(storm_batch* b)
{
    if (!b) return STORM_ERR_INVALID_ARG;
    BK(cudaStreamSynchronize(b->stream));
    return STORM_OK;
}

int storm_batch_get_distribution(storm_batch* b, int i, float* mean, float* sigma)
{
    if (!b || i < 0 || i >= b->n) return STORM_ERR_INVALID_ARG;
    const Problem& pb = b->inst[i].pb;
    if (mean) BK(cudaMemcpyAsync(mean, pb.mu, 4 * pb.H * pb.d, cudaMemcpyDeviceToHost, b->stream));
    if (sigma) BK(cudaMemcpyAsync(sigma, pb.sigma, 4 * pb.d, cudaMemcpyDeviceToHost, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    return STORM_OK;
}

int storm_batch_set_distribution(storm_batch* b, int i, const float* mean, const float* sigma)
{
    if (!b || i < 0 || i >= b->n) return STORM_ERR_INVALID_ARG;
    const Problem& pb = b->inst[i].pb;
    if (mean) BK(cudaMemcpyAsync(pb.mu, mean, 4 * pb.H * pb.d, cudaMemcpyHostToDevice, b->stream));
    if (sigma) BK(cudaMemcpyAsync(pb.sigma, sigma, 4 * pb.d, cudaMemcpyHostToDevice, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    return STORM_OK;
}

int storm_batch_get_launch(const storm_batch* b, int* items, int* threads)
{
    if (!b) return STORM_ERR_INVALID_ARG;
    const bool warp = b->mapping == STORM_MAP_WARP;
    if (items) *items = warp ? 32 * b->wpc : b->items;
    if (threads) *threads = warp ? 32 * b->wpc : b->threads;
    return STORM_OK;
}

int storm_batch_get_launch_mapping(const storm_batch* b) { return b ? b->mapping : STORM_ERR_INVALID_ARG; }

int storm_batch_set_launch(storm_batch* b, int items_per_tile, int threads)
{
    if (!b || threads < 32 || threads > kMaxThreads || threads % 32 || items_per_tile < 1)
        return STORM_ERR_INVALID_ARG;
    BK(cudaStreamSynchronize(b->stream));
    const int rc = batch_apply_launch(b, items_per_tile, threads);
    if (rc) return rc;
    return batch_build_graphs(b);
}

int storm_batch_set_launch_warp(storm_batch* b, int warps_per_cta)
{
    if (!b || warps_per_cta < 1 || warps_per_cta > kWarpMaxWarps) return STORM_ERR_INVALID_ARG;
    BK(cudaStreamSynchronize(b->stream));
    const int rc = batch_apply_launch_warp(b, warps_per_cta);
    if (rc) return rc;
    return batch_build_graphs(b);
}

int storm_batch_autotune(storm_batch* b, float* best_us)
{
    if (!b) return STORM_ERR_INVALID_ARG;
    BK(cudaStreamSynchronize(b->stream));
    const int items_c[] = {32, 48, 64, 96, 128};
    const int threads_c[] = {128, 256, 512};
    const int wpcs[] = {1, 2, 4, 8};
    float best = INFINITY;
    int bm = b->mapping, bi = b->items, bt = b->threads, bw = b->wpc;
    cudaEvent_t e0, e1;
    BK(cudaEventCreate(&e0));
    BK(cudaEventCreate(&e1));
    std::vector<int3> shapes;  // (mapping, items or warps, threads)
    for (int it : items_c)
        for (int th : threads_c) shapes.push_back(make_int3(STORM_MAP_CTA, it, th));
    for (int w : wpcs) shapes.push_back(make_int3(STORM_MAP_WARP, w, 32 * w));
    for (const int3 sh : shapes) {
        const int rc = sh.x == STORM_MAP_WARP ? batch_apply_launch_warp(b, sh.y)
                                              : batch_apply_launch(b, sh.y, sh.z);
        if (rc != STORM_OK) continue;
        std::vector<float> t;
        for (int r = 0; r < 8; ++r) {
            cudaEventRecord(e0, b->stream);
            const cudaError_t le = batch_launch_rollout(b, b->stream, 0);
            cudaEventRecord(e1, b->stream);
            if (le != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                b->err = "autotune launch failed";
                return STORM_ERR_CUDA;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r >= 2) t.push_back(ms * 1e3f);
        }
        std::sort(t.begin(), t.end());
        if (t[t.size() / 2] < best) {
            best = t[t.size() / 2];
            bm = sh.x;
            if (sh.x == STORM_MAP_WARP) {
                bw = sh.y;
            } else {
                bi = sh.y;
                bt = sh.z;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int rc = bm == STORM_MAP_WARP ? batch_apply_launch_warp(b, bw) : batch_apply_launch(b, bi, bt);
    if (rc) return rc;
    if (best_us) *best_us = best;
    return batch_build_graphs(b);
}

}  // extern "C"


// ============================================================================ surrogate C ABI

namespace {
#define MK(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            (void)cudaGetLastError();                                              \
            m->msg = std::string(#call) + ": " + cudaGetErrorString(e_);           \
            return e_ == cudaErrorMemoryAllocation ? STORM_ERR_OOM : STORM_ERR_CUDA; \
        }                                                                          \
    } while (0)

void mlp_free(storm_mlp* m)
{
    mlp_free_buffers(m->buf);
    float* fl[] = {m->p, m->g, m->m, m->v, m->loss, m->th_b, m->t_b, m->loss_hist};
    for (auto* q : fl)
        if (q) cudaFree(q);
    __nv_bfloat16* bf[] = {m->w1, m->w2, m->w2t, m->w3, m->w3t, m->w1p, m->w2p, m->w3p};
    for (auto* q : bf)
        if (q) cudaFree(q);
    if (m->idx) cudaFree(m->idx);
    if (m->err) cudaFree(m->err);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
}

int mlp_check_err(storm_mlp* m)
{
    int e = 0;
    MK(cudaMemcpyAsync(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    MK(cudaStreamSynchronize(m->stream));
    if (e) {
        m->msg = "a tensor-core wait timed out";
        MK(cudaMemsetAsync(m->err, 0, sizeof(int), m->stream));
        return STORM_ERR_TIMEOUT;
    }
    return STORM_OK;
}
}  // namespace

extern "C" {

const char* storm_mlp_last_error(const storm_mlp* m) { return m ? m->msg.c_str() : "NULL network"; }

int storm_mlp_create(uint64_t seed, void* cuda_stream, storm_mlp** out)
{
    return storm_mlp_create_arch(seed, STORM_MLP_DISTANCE, cuda_stream, out);
}

int storm_mlp_param_count(const storm_mlp* m) { return m ? m->a.count : STORM_ERR_INVALID_ARG; }

int storm_mlp_create_arch(uint64_t seed, int arch, void* cuda_stream, storm_mlp** out)
{
    if (!out) return STORM_ERR_INVALID_ARG;
    *out = nullptr;
    if (arch != STORM_MLP_DISTANCE && arch != STORM_MLP_JOINTNERF) return STORM_ERR_INVALID_ARG;
    storm_mlp* m = new (std::nothrow) storm_mlp();
    if (!m) return STORM_ERR_OOM;
    if (arch == STORM_MLP_JOINTNERF) m->a = mlp_arch(1, 256, 128, 64);
    auto fail_m = [&](int rc) {
        fprintf(stderr, "storm_mlp_create: %s\n", m->msg.c_str());
        mlp_free(m);
        delete m;
        return rc;
    };
    int rc = STORM_OK;
    auto try_ = [&](cudaError_t e, const char* what) {
        if (rc == STORM_OK && e != cudaSuccess) {
            (void)cudaGetLastError();
            m->msg = std::string(what) + ": " + cudaGetErrorString(e);
            rc = e == cudaErrorMemoryAllocation ? STORM_ERR_OOM : STORM_ERR_CUDA;
        }
    };
    try_(cudaGetDevice(&m->device), "cudaGetDevice");
    try_(cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, m->device), "SM count");
    try_(cudaFuncSetAttribute(k_mlp_forward_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(tc::kTileSmem)),
         "fused forward shared memory");
    if (cuda_stream) {
        m->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        try_(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking), "stream");
        m->own_stream = rc == STORM_OK;
    }
    const size_t P = sizeof(float) * m->a.count;
    try_(cudaMalloc(&m->p, P), "params");
    try_(cudaMalloc(&m->g, P), "grad");
    try_(cudaMalloc(&m->m, P), "adam m");
    try_(cudaMalloc(&m->v, P), "adam v");
    try_(cudaMalloc(&m->loss, sizeof(float)), "loss");
    try_(cudaMalloc(&m->err, sizeof(int)), "err");
    const size_t hh = sizeof(__nv_bfloat16) * kMlpHid * kMlpHid;
    try_(cudaMalloc(&m->w1, sizeof(__nv_bfloat16) * kMlpHid * kMlpIn), "w1");
    try_(cudaMalloc(&m->w2, hh), "w2");
    try_(cudaMalloc(&m->w2t, hh), "w2t");
    try_(cudaMalloc(&m->w3, hh), "w3");
    try_(cudaMalloc(&m->w3t, hh), "w3t");
    try_(cudaMalloc(&m->w1p, sizeof(__nv_bfloat16) * kMlpHid * kMlpIn), "w1p");
    try_(cudaMalloc(&m->w2p, hh), "w2p");
    try_(cudaMalloc(&m->w3p, hh), "w3p");
    if (rc) return fail_m(rc);
    try_(cudaMemsetAsync(m->m, 0, P, m->stream), "memset");
    try_(cudaMemsetAsync(m->v, 0, P, m->stream), "memset");
    try_(cudaMemsetAsync(m->err, 0, sizeof(int), m->stream), "memset");
    k_mlp_init<<<(m->a.count + 255) / 256, 256, 0, m->stream>>>(
        m->p, m->a, static_cast<uint32_t>(seed & 0xffffffffu), static_cast<uint32_t>(seed >> 32));
    try_(cudaGetLastError(), "init");
    if (rc == STORM_OK) rc = mlp_cast(m, m->stream);
    try_(cudaStreamSynchronize(m->stream), "sync");
    if (rc) return fail_m(rc);
    *out = m;
    return STORM_OK;
}

void storm_mlp_destroy(storm_mlp* m)
{
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    mlp_free(m);
    delete m;
}

int storm_mlp_get_params(storm_mlp* m, float* params)
{
    if (!m || !params) return STORM_ERR_INVALID_ARG;
    MK(cudaMemcpyAsync(params, m->p, sizeof(float) * m->a.count, cudaMemcpyDeviceToHost, m->stream));
    MK(cudaStreamSynchronize(m->stream));
    return STORM_OK;
}

int storm_mlp_set_params(storm_mlp* m, const float* params)
{
    if (!m || !params) return STORM_ERR_INVALID_ARG;
    for (int i = 0; i < m->a.count; ++i)
        if (!std::isfinite(params[i])) return m->msg = "non-finite parameter", STORM_ERR_INVALID_ARG;
    MK(cudaMemcpyAsync(m->p, params, sizeof(float) * m->a.count, cudaMemcpyHostToDevice, m->stream));
    const int rc = mlp_cast(m, m->stream);
    if (rc) return rc;
    MK(cudaStreamSynchronize(m->stream));
    return STORM_OK;
}

int storm_mlp_wait_probe(storm_mlp* m, unsigned int limit_us)
{
    if (!m || limit_us < 1 || limit_us > 1000000) return STORM_ERR_INVALID_ARG;
    tc::k_wait_probe<<<1, tc::kThreads, 0, m->stream>>>(m->err, 1000ull * limit_us);
    MK(cudaGetLastError());
    return mlp_check_err(m);
}

int storm_mlp_predict_async(storm_mlp* m, const float* theta_dev, int count, int dof, float* out_dev)
{
    if (!m || !theta_dev || !out_dev || count < 1 || count > STORM_MLP_MAX_ROWS || dof < 1 || dof > 7)
        return STORM_ERR_INVALID_ARG;
    const int tiles = (count + tc::kBM - 1) / tc::kBM;
    k_mlp_forward_tiles<<<std::min(tiles, m->sms), tc::tile_threads(kFwdEpi), tc::kTileSmem, m->stream>>>(
        mlp_view(m), theta_dev, count, dof, out_dev);
    MK(cudaGetLastError());
    return STORM_OK;
}

int storm_mlp_predict(storm_mlp* m, const float* theta_dev, int count, int dof, float* out_dev)
{
    const int rc = storm_mlp_predict_async(m, theta_dev, count, dof, out_dev);
    return rc ? rc : mlp_check_err(m);
}

int storm_mlp_predict_layers(storm_mlp* m, const float* theta_dev, int count, int dof, float* out_dev)
{
    if (!m || !theta_dev || !out_dev || count < 1 || count > STORM_MLP_MAX_ROWS || dof < 1 || dof > 7)
        return STORM_ERR_INVALID_ARG;
    const int rc = mlp_forward(m, m->buf, theta_dev, count, dof, false, nullptr, m->stream);
    if (rc) return rc;
    MK(cudaMemcpyAsync(out_dev, m->buf.y, sizeof(float) * count, cudaMemcpyDeviceToDevice, m->stream));
    return mlp_check_err(m);
}

int storm_mlp_loss_grad(storm_mlp* m, const float* theta_dev, const float* target_dev, int count,
                        int dof, float* loss, float* grad)
{
    if (!m || !theta_dev || !target_dev || count < 1 || count > STORM_MLP_MAX_ROWS || dof < 1 || dof > 7)
        return STORM_ERR_INVALID_ARG;
    const int R = (count + tc::kBM - 1) / tc::kBM * tc::kBM;
    if (mlp_reserve(m->buf, R, true) != cudaSuccess) return STORM_ERR_OOM;
    int rc = mlp_forward(m, m->buf, theta_dev, count, dof, true, nullptr, m->stream);
    if (!rc) rc = mlp_backward(m, m->buf, target_dev, count, m->stream);
    if (rc) return rc;
    if (loss) MK(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    if (grad) MK(cudaMemcpyAsync(grad, m->g, sizeof(float) * m->a.count, cudaMemcpyDeviceToHost, m->stream));
    return mlp_check_err(m);
}

int storm_mlp_train(storm_mlp* m, const float* theta_dev, const float* target_dev, int count, int dof,
                    int batch, int epochs, float lr, uint64_t seed, float* epoch_loss)
{
    if (!m || !theta_dev || !target_dev || count < batch || batch < 128 || batch % 128 ||
        batch > STORM_MLP_MAX_ROWS || epochs < 1 || !(lr > 0.f) || dof < 1 || dof > 7)
        return STORM_ERR_INVALID_ARG;
    if (mlp_reserve(m->buf, batch, true) != cudaSuccess) return STORM_ERR_OOM;
    const int nb = count / batch;
    if (m->cap_batch < batch) {
        if (m->th_b) cudaFree(m->th_b);
        if (m->t_b) cudaFree(m->t_b);
        m->th_b = m->t_b = nullptr;
        MK(cudaMalloc(&m->th_b, sizeof(float) * batch * 7));
        MK(cudaMalloc(&m->t_b, sizeof(float) * batch));
        m->cap_batch = batch;
    }
    if (m->cap_idx < count) {
        if (m->idx) cudaFree(m->idx);
        m->idx = nullptr;
        MK(cudaMalloc(&m->idx, sizeof(int) * count));
        m->cap_idx = count;
    }
    if (m->cap_hist < nb) {
        if (m->loss_hist) cudaFree(m->loss_hist);
        m->loss_hist = nullptr;
        MK(cudaMalloc(&m->loss_hist, sizeof(float) * nb));
        m->cap_hist = nb;
    }
    std::vector<int> perm(count);
    std::vector<float> hist(nb);
    uint64_t state = seed ^ 0x9E3779B97F4A7C15ull;
    auto next = [&]() {  // splitmix64
        state += 0x9E3779B97F4A7C15ull;
        uint64_t z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    for (int ep = 0; ep < epochs; ++ep) {
        std::iota(perm.begin(), perm.end(), 0);
        for (int i = count - 1; i > 0; --i) std::swap(perm[i], perm[next() % (i + 1)]);
        MK(cudaMemcpyAsync(m->idx, perm.data(), sizeof(int) * count, cudaMemcpyHostToDevice, m->stream));
        MK(cudaStreamSynchronize(m->stream));
        for (int bi = 0; bi < nb; ++bi) {
            k_mlp_gather<<<(batch + 255) / 256, 256, 0, m->stream>>>(theta_dev, target_dev, m->idx, bi * batch,
                                                                   batch, dof, m->th_b, m->t_b);
            int rc = mlp_forward(m, m->buf, m->th_b, batch, dof, true, nullptr, m->stream);
            if (!rc) rc = mlp_backward(m, m->buf, m->t_b, batch, m->stream);
            if (rc) return rc;
            k_adam<<<(m->a.count + 255) / 256, 256, 0, m->stream>>>(m->p, m->g, m->m, m->v, m->a.count, lr,
                                                                   0.9f, 0.999f, 1e-8f, ++m->t);
            rc = mlp_cast(m, m->stream);
            if (rc) return rc;
            MK(cudaMemcpyAsync(m->loss_hist + bi, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, m->stream));
        }
        MK(cudaMemcpyAsync(hist.data(), m->loss_hist, sizeof(float) * nb, cudaMemcpyDeviceToHost, m->stream));
        const int rc = mlp_check_err(m);
        if (rc) return rc;
        if (epoch_loss) {
            double acc = 0.0;
            for (float x : hist) acc += x;
            epoch_loss[ep] = static_cast<float>(acc / nb);
        }
    }
    return STORM_OK;
}

int storm_self_distance(storm_handle* h, const float* theta_dev, int count, float* sd_dev)
{
    if (!h || !theta_dev || !sd_dev || count < 0) return fail(h, STORM_ERR_INVALID_ARG, "bad argument");
    if (count == 0) return STORM_OK;
    const size_t smem = sizeof(float4) * 8 * std::max(h->pb.M, 1);
    k_self_distance<<<(count + 7) / 8, 256, smem, h->stream>>>(h->pb, theta_dev, count, sd_dev);
    CK(cudaGetLastError());
    return STORM_OK;
}

// Self-collision mode (Problem::self_mode) with `mlp`: check the fused kernel's
// shared-memory plan against the device, then re-capture the step graph.
static int set_self_mode(storm_handle* h, storm_mlp* mlp, int mode, double margin)
{
    if (!h || std::isnan(margin)) return fail(h, STORM_ERR_INVALID_ARG, "bad argument");
    CK(cudaStreamSynchronize(h->stream));
    if (mlp) {
        if (mlp->device != h->device) return fail(h, STORM_ERR_INVALID_ARG, "network on another device");
        const MlpRolloutPlan P = mlp_rollout_plan(h->pb);
        int optin = 0;
        CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
        for (auto kf : {k_rollout_mlp<false>, k_rollout_mlp<true>}) {
            cudaFuncAttributes fa;
            CK(cudaFuncGetAttributes(&fa, kf));
            if (static_cast<size_t>(P.bytes) + fa.sharedSizeBytes > static_cast<size_t>(optin))
                return fail(h, STORM_ERR_INVALID_ARG, "problem too large for the fused network rollout");
            CK(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    optin - static_cast<int>(fa.sharedSizeBytes)));
        }
        h->mlp_smem = P.bytes;
        // the network's own stream may still be writing its weights
        CK(cudaStreamSynchronize(mlp->stream));
    }
    h->mlp = mlp;
    h->pb.self_mode = mlp ? mode : 0;
    h->pb.self_margin = static_cast<float>(margin);
    return build_graphs(h);
}

int storm_set_surrogate_cost(storm_handle* h, storm_mlp* mlp) { return set_self_mode(h, mlp, 2, 0.0); }

int storm_set_surrogate(storm_handle* h, storm_mlp* mlp, double margin)
{
    return set_self_mode(h, mlp, 1, margin);
}

}  // extern "C"
