// storm_adjoint.cuh -- adjoint of the rollout cost with respect to the mean.
//
// The paper optimises the mean by sampling only; this kernel adds the exact
// gradient of J(mu) = (1/N) sum_n C_hat_n(mu + sigma o eps~_n) with the noise
// fixed, back through the running cost (Eqs. 9-15), the kinematics (Eq. 8)
// and the integration scan (Eq. 7).  Kinks take the zero subgradient, the
// collision minimum follows its minimiser, and the manipulability indicator
// is differentiated only where m < k_m.  Included by storm.cu after the
// rollout kernel.
#pragma once

struct AdjointLayout {
    int frame, cent, sph, wsph, boxlh, pblk, keyw, keys;                 // 16/8-byte arrays
    int lb, lcent, mask, lcap;                                           // broad phase
    int mu, sigma, eps, u, th, thd, basis, dt, gpow, vmax, dhx, qlo, qhi;  // float arrays
    int boxes, cost, goal, state, gth, gthd, gu, gup;
    int first, slink, pairs;
    int bytes;
};

// Float4s per step of the frame array: the F x 3 rows of its link frames, padded
// to an odd count so that the threads of a warp, one step each, read their
// frames from different shared-memory banks.
__host__ __device__ inline int adjoint_frame_stride(const Problem& pb)
{
    const int r = (pb.d + 1) * 3;
    return r + ((r & 1) ? 0 : 1);
}

__host__ __device__ inline AdjointLayout adjoint_layout(const Problem& pb)
{
    AdjointLayout L;
    int off = 0;
    const int I = pb.H;  // one particle per CTA
    L.frame = take_(off, I * adjoint_frame_stride(pb) * 16);
    L.cent = take_(off, I * pb.M * 16);
    L.sph = take_(off, pb.M * 16);
    L.wsph = take_(off, pb.O * 16);
    L.boxlh = take_(off, pb.B * 2 * 16);
    L.pblk = take_(off, pb.NPB * 16);
    L.keyw = take_(off, I * 8);
    L.keys = take_(off, I * 8);
    L.lb = take_(off, (pb.d + 1) * 16);         // link bounding spheres (local centre, radius)
    L.lcent = take_(off, I * (pb.d + 1) * 16);  // their centres per step
    L.mask = take_(off, I * (pb.d + 1) * 16);   // per (step, frame): boxes, obstacle spheres met
    L.lcap = take_(off, 2 * (pb.d + 1) * 16);   // link capsules (local ends, radius)
    L.mu = take_(off, pb.H * pb.d * 4);
    L.sigma = take_(off, pb.d * 4);
    L.eps = take_(off, pb.S * pb.d * 4);
    L.u = take_(off, pb.H * pb.d * 4);
    L.th = take_(off, pb.H * pb.d * 4);
    L.thd = take_(off, pb.H * pb.d * 4);
    L.basis = take_(off, pb.spline ? pb.H * pb.S * 4 : 0);
    L.dt = take_(off, pb.H * 4);
    L.gpow = take_(off, pb.H * 4);
    L.vmax = take_(off, pb.H * 4);
    L.dhx = take_(off, pb.d * 8 * 4);
    L.qlo = take_(off, pb.d * 4);
    L.qhi = take_(off, pb.d * 4);
    L.boxes = take_(off, pb.B * 6 * 4);
    L.cost = take_(off, I * 4);
    L.goal = take_(off, 12 * 4);
    L.state = take_(off, 3 * pb.d * 4);
    L.gth = take_(off, I * pb.d * 4);
    L.gthd = take_(off, I * pb.d * 4);
    L.gu = take_(off, I * pb.d * 4);
    L.gup = take_(off, I * pb.d * 4);
    L.first = take_(off, (pb.d + 2) * 4);
    L.slink = take_(off, pb.M * 4);
    L.pairs = take_(off, pb.P * 4);
    L.bytes = off;
    return L;
}

// A point of a link frame in world coordinates (the frame's three [R | p] rows).
__device__ __forceinline__ float3 frame_apply(const float4* T, float4 q)
{
    const float4 r0 = T[0], r1 = T[1], r2 = T[2];
    return make_float3(fmaf(r0.x, q.x, fmaf(r0.y, q.y, fmaf(r0.z, q.z, r0.w))),
                       fmaf(r1.x, q.x, fmaf(r1.y, q.y, fmaf(r1.z, q.z, r1.w))),
                       fmaf(r2.x, q.x, fmaf(r2.y, q.y, fmaf(r2.z, q.z, r2.w))));
}

// Minimiser ids of a pair block: (first-link sphere - first) * 8 + second-link
// slot, below 64 * 8 = 512 for up to 64 spheres on the first link; the
// leftover pairs' ids start at 2^24, above every block's.
constexpr uint32_t kSelfBlockIds = 512;

__device__ __forceinline__ unsigned long long depth_key(float depth, uint32_t idx)
{
    return (static_cast<unsigned long long>(__float_as_uint(depth)) << 32) | (0xffffffffu - idx);
}

// w * g^T dc/dtheta for a point c rigidly attached to frame f (joints 0..f-1
// move it: dc/dtheta_k = z_k x (c - o_k), z_k / o_k of frame k + 1).
__device__ __forceinline__ void add_point_grad(const float4* fr, int f, float cx, float cy, float cz,
                                               float gx, float gy, float gz, float w,
                                               float (&gth)[kMaxDof])
{
#pragma unroll
    for (int k = 0; k < kMaxDof; ++k) {
        if (k < f) {
            const float4 r0 = fr[(k + 1) * 3 + 0], r1 = fr[(k + 1) * 3 + 1], r2 = fr[(k + 1) * 3 + 2];
            const float zx = r0.z, zy = r1.z, zz = r2.z;
            const float rx = cx - r0.w, ry = cy - r1.w, rz = cz - r2.w;
            const float vx = zy * rz - zz * ry, vy = zz * rx - zx * rz, vz = zx * ry - zy * rx;
            gth[k] = fmaf(w, gx * vx + gy * vy + gz * vz, gth[k]);
        }
    }
}

// The sums of grad = (1/N) sum_{n >= n_null} dC_n/du_n and J = (1/N) sum_n C_n,
// kept in 64-bit fixed point: integer additions give the same bits in any
// order, so the particles' CTAs add their rows with atomics and the result is
// still deterministic (and, with 2^-30 resolution per gradient entry and 2^-20
// per cost, finer than an FP32 sum).  Zero between launches (the CTA that
// finishes a launch clears them).
struct AdjAcc {
    unsigned long long* sum;  // H*d gradient sums, then the cost sum
    unsigned int* count;      // CTAs that have added their row this launch
    int* bad;                 // a non-finite or out-of-range value was seen
};

constexpr double kAdjGradScale = 1073741824.0;  // 2^30
constexpr double kAdjCostScale = 1048576.0;     // 2^20

__device__ __forceinline__ void adj_add(unsigned long long* sum, float v, double scale, int* bad)
{
    const double x = static_cast<double>(v) * scale;
    if (!(fabs(x) < 4.0e18 / 16384.0)) {  // NaN, infinite, or a sum of up to 2^14 rows that could overflow
        atomicExch(bad, 1);
        return;
    }
    atomicAdd(sum, static_cast<unsigned long long>(__double2ll_rn(x)));
}

// One particle per CTA: forward rollout, per-step gradients, reverse scans,
// then the CTA adds its dC/du row and C to the fixed-point sums; the CTA that
// arrives last turns them into grad and J (and with eta != 0 steps
// mu <- mu - eta grad; with `finalize` the control step ends there: the command
// from the refined mean, the step counter advanced).  A non-finite value makes
// grad and J NaN and leaves mu as it was.
__global__ void __launch_bounds__(128)
k_adjoint(Problem pb, const float* __restrict__ mean, const float* __restrict__ state,
          const float* __restrict__ goal, StepState* st, int step_override,
          int iter, AdjAcc acc, float* __restrict__ Ctot, float* __restrict__ grad_out,
          float* __restrict__ J_out, float eta, float* __restrict__ cmd_out, int finalize)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const AdjointLayout L = adjoint_layout(pb);
    float4* s_frame = reinterpret_cast<float4*>(smem + L.frame);
    float4* s_cent = reinterpret_cast<float4*>(smem + L.cent);
    float4* s_sph = reinterpret_cast<float4*>(smem + L.sph);
    float4* s_wsph = reinterpret_cast<float4*>(smem + L.wsph);
    float4* s_boxlh = reinterpret_cast<float4*>(smem + L.boxlh);
    uint4* s_pblk = reinterpret_cast<uint4*>(smem + L.pblk);
    unsigned long long* s_keyw = reinterpret_cast<unsigned long long*>(smem + L.keyw);
    unsigned long long* s_keys = reinterpret_cast<unsigned long long*>(smem + L.keys);
    float4* s_lb = reinterpret_cast<float4*>(smem + L.lb);
    float4* s_lcent = reinterpret_cast<float4*>(smem + L.lcent);
    unsigned long long* s_mask = reinterpret_cast<unsigned long long*>(smem + L.mask);
    float4* s_lcap = reinterpret_cast<float4*>(smem + L.lcap);
    float* s_mu = reinterpret_cast<float*>(smem + L.mu);
    float* s_sigma = reinterpret_cast<float*>(smem + L.sigma);
    float* s_eps = reinterpret_cast<float*>(smem + L.eps);
    float* s_u = reinterpret_cast<float*>(smem + L.u);
    float* s_th = reinterpret_cast<float*>(smem + L.th);
    float* s_thd = reinterpret_cast<float*>(smem + L.thd);
    float* s_basis = reinterpret_cast<float*>(smem + L.basis);
    float* s_dt = reinterpret_cast<float*>(smem + L.dt);
    float* s_gpow = reinterpret_cast<float*>(smem + L.gpow);
    float* s_vmax = reinterpret_cast<float*>(smem + L.vmax);
    float* s_dhx = reinterpret_cast<float*>(smem + L.dhx);
    float* s_qlo = reinterpret_cast<float*>(smem + L.qlo);
    float* s_qhi = reinterpret_cast<float*>(smem + L.qhi);
    float* s_boxes = reinterpret_cast<float*>(smem + L.boxes);
    float* s_cost = reinterpret_cast<float*>(smem + L.cost);
    float* s_goal = reinterpret_cast<float*>(smem + L.goal);
    float* s_state = reinterpret_cast<float*>(smem + L.state);
    float* s_gth = reinterpret_cast<float*>(smem + L.gth);
    float* s_gthd = reinterpret_cast<float*>(smem + L.gthd);
    float* s_gu = reinterpret_cast<float*>(smem + L.gu);
    float* s_gup = reinterpret_cast<float*>(smem + L.gup);
    int* s_first = reinterpret_cast<int*>(smem + L.first);
    int* s_slink = reinterpret_cast<int*>(smem + L.slink);
    uint32_t* s_pairs = reinterpret_cast<uint32_t*>(smem + L.pairs);

    const int tid = threadIdx.x, nt = blockDim.x;
    const int d = pb.d, H = pb.H, S = pb.S, M = pb.M, F = pb.d + 1, HD = pb.H * pb.d;
    const int FS = adjoint_frame_stride(pb);
    const int n = blockIdx.x, I = H;
    const uint32_t step = step_override >= 0 ? static_cast<uint32_t>(step_override) : st->step;
    const int NO = pb.B + pb.O;

    // ---- stage: every table this CTA reads, as asynchronous copies issued at
    // once (they land while the noise is drawn); the goal goes through s_cost,
    // which the cost phase overwrites later
    {
        auto cp4 = [](void* dst, const void* src) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(dst))),
                         "l"(src)
                         : "memory");
        };
        auto cp16 = [](void* dst, const void* src) {
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(dst))),
                         "l"(src)
                         : "memory");
        };
        for (int i = tid; i < HD; i += nt) cp4(s_mu + i, mean + i);
        for (int i = tid; i < d; i += nt) {
            cp4(s_sigma + i, pb.sigma + i);
            cp4(s_qlo + i, pb.qlo + i);
            cp4(s_qhi + i, pb.qhi + i);
        }
        for (int i = tid; i < 3 * d; i += nt) cp4(s_state + i, state + i);
        for (int i = tid; i < 7; i += nt) cp4(s_cost + i, goal + i);
        for (int i = tid; i < H; i += nt) {
            cp4(s_dt + i, pb.dt + i);
            cp4(s_gpow + i, pb.gpow + i);
            cp4(s_vmax + i, pb.vmax + i);
        }
        if (pb.spline)
            for (int i = tid; i < H * S; i += nt) cp4(s_basis + i, pb.basis + i);
        for (int i = tid; i < d * 8; i += nt) cp4(s_dhx + i, pb.dhx + i);
        for (int i = tid; i < d + 2; i += nt) cp4(s_first + i, pb.link_first + i);
        for (int i = tid; i < F; i += nt) cp16(s_lb + i, pb.lbound + i);
        for (int i = tid; i < 2 * F; i += nt) cp16(s_lcap + i, pb.lcap + i);
        for (int i = tid; i < M; i += nt) cp16(s_sph + i, pb.sph + i);
        for (int i = tid; i < pb.P; i += nt) cp4(s_pairs + i, pb.pairs + i);
        for (int i = tid; i < pb.NPB; i += nt) cp16(s_pblk + i, pb.pblk + i);
        for (int i = tid; i < 6 * pb.B; i += nt) cp4(s_boxes + i, pb.boxes + i);
        for (int i = tid; i < pb.O; i += nt) cp16(s_wsph + i, pb.wsph + i);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    __shared__ int s_task_v;
    __shared__ float s_ubox[4][6];  // the collision warps' boxes around the CTA's link bounds
    __shared__ unsigned s_cand[4];  // obstacles that box meets: boxes 0-31, 32-63, spheres 0-31, 32-63
    __shared__ int s_cflag_v;
    int* s_task = &s_task_v;
    volatile int* s_cflag = &s_cflag_v;
    if (tid == 0) {
        s_task_v = 0;
        s_cflag_v = 0;
    }
    for (int i = tid; i < H; i += nt) {
        s_keyw[i] = 0ull;
        s_keys[i] = 0ull;
    }
    // ---- noise of particle n (same stream as the rollout)
    const int per = S * d;
    if (pb.sampler == STORM_SAMPLER_PHILOX) {
        const uint32_t e0 = static_cast<uint32_t>(n) * per, e1 = e0 + per;
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
        for (int i = tid; i < per; i += nt) s_eps[i] = pb.halton[static_cast<size_t>(n) * per + i];
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    // ---- derived tables: sphere -> frame, box bounds, the goal rotation
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
    if (tid == 0) {
        const float* goal_s = s_cost;
        const float qn = rsqrtf(goal_s[3] * goal_s[3] + goal_s[4] * goal_s[4] + goal_s[5] * goal_s[5] +
                                goal_s[6] * goal_s[6]);
        const float w = goal_s[3] * qn, x = goal_s[4] * qn, y = goal_s[5] * qn, z = goal_s[6] * qn;
        float gr[12];
        gr[0] = 1.f - 2.f * (y * y + z * z);
        gr[1] = 2.f * (x * y - w * z);
        gr[2] = 2.f * (x * z + w * y);
        gr[3] = 2.f * (x * y + w * z);
        gr[4] = 1.f - 2.f * (x * x + z * z);
        gr[5] = 2.f * (y * z - w * x);
        gr[6] = 2.f * (x * z - w * y);
        gr[7] = 2.f * (y * z + w * x);
        gr[8] = 1.f - 2.f * (x * x + y * y);
        gr[9] = goal_s[0];
        gr[10] = goal_s[1];
        gr[11] = goal_s[2];
#pragma unroll
        for (int k = 0; k < 12; ++k) s_goal[k] = gr[k];
    }
    for (int i = tid; i < HD; i += nt) {
        const int h = i / d, j = i - h * d;
        float e;
        if (pb.spline) {
            e = 0.f;
            for (int s = 0; s < S; ++s) e = fmaf(s_basis[h * S + s], s_eps[s * d + j], e);
        } else {
            e = s_eps[h * d + j];
        }
        s_u[i] = (n < pb.n_null) ? 0.f : fmaf(s_sigma[j], e, s_mu[i]);
    }
    __syncthreads();
    for (int j = tid; j < d; j += nt) {
        float v = s_state[d + j], q = s_state[j];
#pragma unroll 6
        for (int h = 0; h < H; ++h) {  // (unrolled: later steps' loads issue ahead of the scan)
            v = fmaf(s_dt[h], s_u[h * d + j], v);
            q = fmaf(s_dt[h], v, q);
            s_thd[h * d + j] = v;
            s_th[h * d + j] = q;
        }
    }
    __syncthreads();

    // ---- per step h: FK frames
    for (int h = tid; h < I; h += nt) {
        const float* th = s_th + h * d;
        float4* fr = s_frame + h * FS;
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
    }
    __syncthreads();

    // From here two groups of warps work side by side until the next CTA
    // barrier: the first ceil(I / 32) warps take the non-collision costs and
    // their gradients, one step per thread; the others the collision broad
    // phase and the world and self minimisers (their own named barrier between
    // passes).  Neither reads what the other writes.
    const int cost_warps = (I + 31) / 32;
    const int coll_threads = nt - cost_warps * 32;  // > 0: I <= 64 < nt / 32 * 32 - 32
    const bool cost_warp = tid < cost_warps * 32;
    const int ct = tid - cost_warps * 32;  // collision thread index
    auto coll_sync = [&]() { asm volatile("bar.sync 1, %0;" ::"r"(coll_threads) : "memory"); };
    const bool bp = pb.broadphase != 0;
    // the self-collision tasks: (step, pair block) dealt a warp's worth at a
    // time; the blocks whose link bounds overlap are taken four at a time, eight
    // lanes each (lane r of a group tests the block's first-link spheres r, r + 8,
    // ... against its second-link spheres), so that the exact tests are spread
    // over the warp instead of one lane per block
    auto coll_self_tasks = [&]() {
        const int lane = tid & 31, ntask = I * pb.NPB;
        const int grp = lane >> 3, r8 = lane & 7;
        // task -> step without a division: (task + 1/2) / NPB is at least 1/(2 NPB)
        // from an integer, far beyond FP32's error for the task counts here
        const float inv_npb = 1.f / static_cast<float>(pb.NPB > 0 ? pb.NPB : 1);
        auto step_of = [&](int task) { return __float2int_rd((static_cast<float>(task) + 0.5f) * inv_npb); };
        while (true) {
            int base = 0;
            if (lane == 0) base = atomicAdd(s_task, 32);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base >= ntask) break;
            const int idx = base + lane;
            bool live = idx < ntask;
            if (live && bp) {  // the two links' bounds apart: no pair of the block touches
                const int item = step_of(idx);
                const uint4 blk = s_pblk[idx - item * pb.NPB];
                const float4 A = s_lcent[item * F + s_slink[blk.x]], B2 = s_lcent[item * F + s_slink[blk.z]];
                const float ex = A.x - B2.x, ey = A.y - B2.y, ez = A.z - B2.z;
                const float rr = A.w + B2.w;
                live = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < rr * rr;
                if (live) {  // the bounding spheres meet: do the links' capsules?
                    const int fa = s_slink[blk.x], fb = s_slink[blk.z];
                    const float4 a0 = s_lcap[2 * fa], a1 = s_lcap[2 * fa + 1];
                    const float4 b0 = s_lcap[2 * fb], b1 = s_lcap[2 * fb + 1];
                    const float4* Ta = s_frame + item * FS + fa * 3;
                    const float4* Tb = s_frame + item * FS + fb * 3;
                    const float rc = a0.w + b0.w;
                    live = seg_seg_dist2(frame_apply(Ta, a0), frame_apply(Ta, a1), frame_apply(Tb, b0),
                                         frame_apply(Tb, b1)) < rc * rc;
                }
            }
            unsigned alive = __ballot_sync(0xffffffffu, live);
            while (alive) {
                const unsigned src = __fns(alive, 0, grp + 1);  // this group's block: the (grp+1)-th live lane
                const int tix = __shfl_sync(0xffffffffu, idx, static_cast<int>(src & 31u));
                unsigned long long key = 0ull;
                int item = 0;
                if (src != 0xffffffffu) {
                    item = step_of(tix);
                    const int bk = tix - item * pb.NPB;
                    const uint4 blk = s_pblk[bk];
                    const float4* ci = s_cent + item * M;
                    float4 cb[8];  // the block's second-link spheres (absent ones far away)
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        cb[k] = k < static_cast<int>(blk.w) ? ci[blk.z + k] : make_float4(1e30f, 1e30f, 1e30f, 0.f);
                    float depth = 0.f;
                    int best = -1;
                    for (uint32_t a = blk.x + r8; a < blk.y; a += 8) {
                        const float4 ca = ci[a];
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const float ex = ca.x - cb[k].x, ey = ca.y - cb[k].y, ez = ca.z - cb[k].z;
                            const float dist2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                            const float rs = ca.w + cb[k].w;
                            if (dist2 < rs * rs && rs - sqrtf(dist2) > depth) {
                                depth = rs - sqrtf(dist2);
                                best = static_cast<int>((a - blk.x) * 8 + k);
                            }
                        }
                    }
                    if (best >= 0) key = depth_key(depth, static_cast<uint32_t>(bk * kSelfBlockIds + best));
                }
#pragma unroll
                for (int o = 4; o > 0; o >>= 1) {  // the group's deepest pair (lowest id on a tie)
                    const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
                    key = other > key ? other : key;
                }
                if (r8 == 0 && key) atomicMax(s_keys + item, key);
#pragma unroll
                for (int g = 0; g < 4; ++g) alive &= alive - 1u;  // the four blocks just taken
            }
        }
    };

    // ---- per step h: non-collision costs and their gradients
    for (int h = tid; cost_warp && h < I; h += cost_warps * 32) {
        const float* th = s_th + h * d;
        const float* thd = s_thd + h * d;
        const float* uh = s_u + h * d;
        const float* up = (h == 0) ? s_state + 2 * d : uh - d;
        const float4* fr = s_frame + h * FS;
        float R[9], pp[3];  // the end effector's frame
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float4 q = fr[d * 3 + r];
            R[r * 3 + 0] = q.x, R[r * 3 + 1] = q.y, R[r * 3 + 2] = q.z, pp[r] = q.w;
        }
        GramFactor G;  // J J^T of the geometric Jacobian, column by column in joint order
        G.zero();
#pragma unroll
        for (int i = 0; i < kMaxDof; ++i) {
            if (i < d) {
                const float4 r0 = fr[(i + 1) * 3], r1 = fr[(i + 1) * 3 + 1], r2 = fr[(i + 1) * 3 + 2];
                const float zx = r0.z, zy = r1.z, zz = r2.z;
                float x[6] = {r1.w * zz - r2.w * zy, r2.w * zx - r0.w * zz, r0.w * zy - r1.w * zx, zx, zy, zz};
                G.add(x);
            }
        }
        float gth[kMaxDof], gthd[kMaxDof], gu[kMaxDof], gup[kMaxDof];
#pragma unroll
        for (int k = 0; k < kMaxDof; ++k) gth[k] = gthd[k] = gu[k] = gup[k] = 0.f;
        const float* Rg = s_goal;
        // position
        const float dx = pp[0] - Rg[9], dy = pp[1] - Rg[10], dz = pp[2] - Rg[11];
        float e[3], c_pos = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            e[a] = pb.pos_w[a] * fmaf(Rg[a], dx, fmaf(Rg[3 + a], dy, Rg[6 + a] * dz));
            c_pos = fmaf(e[a], e[a], c_pos);
        }
        c_pos = sqrtf(c_pos);
        float gp[3] = {0.f, 0.f, 0.f};
        if (c_pos > 0.f) {
#pragma unroll
            for (int r = 0; r < 3; ++r)
                gp[r] = (Rg[r * 3 + 0] * pb.pos_w[0] * e[0] + Rg[r * 3 + 1] * pb.pos_w[1] * e[1] +
                         Rg[r * 3 + 2] * pb.pos_w[2] * e[2]) / c_pos;
        }
        // rotation: d tr(A [w]x) with A built per mode
        float c_rot = 0.f, gw[3] = {0.f, 0.f, 0.f};
        if (pb.rot_mode == STORM_ROT_QUAT) {
            float tr = 0.f;
#pragma unroll
            for (int k = 0; k < 9; ++k) tr = fmaf(Rg[k], R[k], tr);
            const float s1 = sqrtf(fmaxf(0.f, 1.f + tr));
            c_rot = 1.f - 0.5f * s1;
            if (s1 > 0.f) {
                float A[9];  // R_ee R_g^T
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        A[r * 3 + c] = R[r * 3 + 0] * Rg[c * 3 + 0] + R[r * 3 + 1] * Rg[c * 3 + 1] +
                                       R[r * 3 + 2] * Rg[c * 3 + 2];
                const float f = -0.25f / s1;
                gw[0] = f * (A[5] - A[7]);
                gw[1] = f * (A[6] - A[2]);
                gw[2] = f * (A[1] - A[3]);
            }
        } else {
            float E[9];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float rtr = Rg[r] * R[c] + Rg[3 + r] * R[3 + c] + Rg[6 + r] * R[6 + c];
                    E[r * 3 + c] = ((r == c) ? 1.f : 0.f) - rtr;
                    const float we = E[r * 3 + c] * pb.rot_w[c];
                    c_rot = fmaf(we, we, c_rot);
                }
            c_rot = sqrtf(c_rot);
            if (c_rot > 0.f) {
                float Mt[9], T[9], A[9];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int q = 0; q < 3; ++q) Mt[q * 3 + r] = E[r * 3 + q] * pb.rot_w[q] * pb.rot_w[q];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        T[r * 3 + q] = R[r * 3 + 0] * Mt[0 * 3 + q] + R[r * 3 + 1] * Mt[1 * 3 + q] +
                                       R[r * 3 + 2] * Mt[2 * 3 + q];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        A[r * 3 + q] = T[r * 3 + 0] * Rg[q * 3 + 0] + T[r * 3 + 1] * Rg[q * 3 + 1] +
                                       T[r * 3 + 2] * Rg[q * 3 + 2];
                gw[0] = -(A[5] - A[7]) / c_rot;
                gw[1] = -(A[6] - A[2]) / c_rot;
                gw[2] = -(A[1] - A[3]) / c_rot;
            }
        }
        // pose gradients through the geometric Jacobian about the end effector
#pragma unroll
        for (int k = 0; k < kMaxDof; ++k) {
            if (k < d) {
                const float4 r0 = fr[(k + 1) * 3], r1 = fr[(k + 1) * 3 + 1], r2 = fr[(k + 1) * 3 + 2];
                const float zx = r0.z, zy = r1.z, zz = r2.z;
                const float rx = pp[0] - r0.w, ry = pp[1] - r1.w, rz = pp[2] - r2.w;
                const float jx = zy * rz - zz * ry, jy = zz * rx - zx * rz, jz = zx * ry - zy * rx;
                gth[k] += pb.w_pos * (gp[0] * jx + gp[1] * jy + gp[2] * jz) +
                          pb.w_rot * (gw[0] * zx + gw[1] * zy + gw[2] * zz);
            }
        }
        // stop, joint limits, smoothness
        float c_stop = 0.f, c_joint = 0.f, c_smooth = 0.f;
        const float vlim = s_vmax[h];
        float vs[kMaxDof], vj[kMaxDof];
#pragma unroll
        for (int j = 0; j < kMaxDof; ++j) {
            vs[j] = vj[j] = 0.f;
            if (j < d) {
                vs[j] = fmaxf(0.f, fabsf(thd[j]) - vlim);
                c_stop = fmaf(vs[j], vs[j], c_stop);
                vj[j] = fmaxf(0.f, s_qlo[j] - th[j]) + fmaxf(0.f, th[j] - s_qhi[j]);
                c_joint = fmaf(vj[j], vj[j], c_joint);
                const float du = uh[j] - up[j];
                c_smooth = fmaf(du, du, c_smooth);
                gu[j] += pb.w_smooth * 2.f * du;
                gup[j] -= pb.w_smooth * 2.f * du;
            }
        }
        c_stop = sqrtf(c_stop);
        c_joint = sqrtf(c_joint);
#pragma unroll
        for (int j = 0; j < kMaxDof; ++j) {
            if (j < d) {
                if (c_stop > 0.f && vs[j] > 0.f)
                    gthd[j] += pb.w_stop * vs[j] * (thd[j] > 0.f ? 1.f : -1.f) / c_stop;
                if (c_joint > 0.f && vj[j] > 0.f)
                    gth[j] += pb.w_joint * vj[j] * (th[j] < s_qlo[j] ? -1.f : 1.f) / c_joint;
            }
        }
        // manipulability: dm/dtheta_k = m tr(J0^+ dJ0/dtheta_k), J0 about the base origin;
        // J0^+ columns from the Givens factor R (R^T R = J0 J0^T): solve R^T y = J0_i, R x = y
        const float m = G.sqrt_det();
        float c_manip = 0.f;
        if (m < pb.k_m) {
            c_manip = 1.f - m;
            if (m > 0.f && pb.w_manip != 0.f) {
                // column i of J0^+ (6 values, then dropped) contributes to tr_k for every k < i;
                // each tr_k is still summed over i in ascending order
                float tr[kMaxDof], inv_r[6];  // the factor's diagonal, inverted once for the solves
#pragma unroll
                for (int k = 0; k < kMaxDof; ++k) tr[k] = 0.f;
#pragma unroll
                for (int a = 0; a < 6; ++a) inv_r[a] = 1.f / G.r[GramFactor::at(a, a)];
#pragma unroll
                for (int i = 0; i < kMaxDof; ++i) {
                    if (i < d) {
                        const float4 a0 = fr[(i + 1) * 3], a1 = fr[(i + 1) * 3 + 1], a2 = fr[(i + 1) * 3 + 2];
                        float x[6] = {a1.w * a2.z - a2.w * a1.z, a2.w * a0.z - a0.w * a2.z,
                                      a0.w * a1.z - a1.w * a0.z, a0.z, a1.z, a2.z};
                        float y[6], jp[6];
#pragma unroll
                        for (int a = 0; a < 6; ++a) {  // R^T y = x (R^T lower triangular)
                            float sacc = x[a];
#pragma unroll
                            for (int b = 0; b < a; ++b) sacc = fmaf(-G.r[GramFactor::at(b, a)], y[b], sacc);
                            y[a] = sacc * inv_r[a];
                        }
#pragma unroll
                        for (int a = 5; a >= 0; --a) {  // R jp = y
                            float sacc = y[a];
#pragma unroll
                            for (int b = a + 1; b < 6; ++b) sacc = fmaf(-G.r[GramFactor::at(a, b)], jp[b], sacc);
                            jp[a] = sacc * inv_r[a];
                        }
#pragma unroll
                        for (int k = 0; k < kMaxDof; ++k) {
                            if (k < i) {
                                const float4 k0 = fr[(k + 1) * 3], k1 = fr[(k + 1) * 3 + 1], k2 = fr[(k + 1) * 3 + 2];
                                // dz = z_k x z_i ; do = z_k x (o_i - o_k)
                                const float dzx = k1.z * a2.z - k2.z * a1.z, dzy = k2.z * a0.z - k0.z * a2.z,
                                            dzz = k0.z * a1.z - k1.z * a0.z;
                                const float rx = a0.w - k0.w, ry = a1.w - k1.w, rz = a2.w - k2.w;
                                const float dox = k1.z * rz - k2.z * ry, doy = k2.z * rx - k0.z * rz,
                                            doz = k0.z * ry - k1.z * rx;
                                // d(o x z) = do x z + o x dz
                                const float vx = (doy * a2.z - doz * a1.z) + (a1.w * dzz - a2.w * dzy);
                                const float vy = (doz * a0.z - dox * a2.z) + (a2.w * dzx - a0.w * dzz);
                                const float vz = (dox * a1.z - doy * a0.z) + (a0.w * dzy - a1.w * dzx);
                                tr[k] += jp[0] * vx + jp[1] * vy + jp[2] * vz + jp[3] * dzx + jp[4] * dzy + jp[5] * dzz;
                            }
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < kMaxDof; ++k)
                    if (k < d) gth[k] -= pb.w_manip * m * tr[k];
            }
        }
        s_cost[h] = pb.w_pos * c_pos + pb.w_rot * c_rot + pb.w_stop * c_stop + pb.w_joint * c_joint +
                    pb.w_manip * c_manip + pb.w_smooth * c_smooth;
#pragma unroll
        for (int j = 0; j < kMaxDof; ++j) {
            if (j < d) {
                s_gth[h * d + j] = gth[j];
                s_gthd[h * d + j] = gthd[j];
                s_gu[h * d + j] = gu[j];
                s_gup[h * d + j] = gup[j];
            }
        }
    }

    if (cost_warp) {  // the cost warp: join the self-collision tasks once they are open (bounded wait)
        auto now = []() {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            return t;
        };
        bool open = false;
        if ((tid & 31) == 0) {
            open = *s_cflag != 0;
            const unsigned long long t0 = open ? 0ull : now();
            for (uint32_t k = 1; !open; ++k) {
                open = *s_cflag != 0;
                if (!open && (k & 63u) == 0u && now() - t0 > 100000ull) break;  // 100 us: then leave it to them
            }
        }
        open = __shfl_sync(0xffffffffu, open, 0);
        __threadfence_block();  // (acquire: the centres and bounds written before the flag)
        if (open) coll_self_tasks();
    }
    // ---- broad phase (as in the rollout kernels): each step's link-bound centres
    // and, per (step, frame), the boxes and obstacle spheres its bound meets.  A
    // sphere can only touch what its link's bound touches, so the exact tests
    // below skip nothing that penetrates: the same depths and minimisers.
    const unsigned long long all_b = pb.B >= 64 ? ~0ull : (1ull << pb.B) - 1ull;
    const unsigned long long all_o = pb.O >= 64 ? ~0ull : (1ull << pb.O) - 1ull;
    if (!cost_warp) {  // the collision warps
    if (bp) {
        // the bounds' centres, and one box around every bound of the CTA's steps;
        // the obstacles that box meets are the only candidates for any (step,
        // frame) below (a conservative cull: the same masks as testing all)
        float ulo[3] = {INFINITY, INFINITY, INFINITY}, uhi[3] = {-INFINITY, -INFINITY, -INFINITY};
        const int bp_dq = coll_threads / F, bp_dr = coll_threads - bp_dq * F;
        int bp_item = ct / F, bp_f = ct - bp_item * F;
        for (int idx = ct; idx < I * F; idx += coll_threads) {
            const int item = bp_item, f = bp_f;
            bp_item += bp_dq, bp_f += bp_dr;
            if (bp_f >= F) bp_f -= F, ++bp_item;
            const float4 q = s_lb[f];
            const float4* T = s_frame + item * FS + f * 3;
            const float4 r0 = T[0], r1 = T[1], r2 = T[2];
            const float cx = fmaf(r0.x, q.x, fmaf(r0.y, q.y, fmaf(r0.z, q.z, r0.w)));
            const float cy = fmaf(r1.x, q.x, fmaf(r1.y, q.y, fmaf(r1.z, q.z, r1.w)));
            const float cz = fmaf(r2.x, q.x, fmaf(r2.y, q.y, fmaf(r2.z, q.z, r2.w)));
            s_lcent[idx] = make_float4(cx, cy, cz, q.w);
            if (q.w > 0.f) {  // (a frame without spheres has an empty bound)
                ulo[0] = fminf(ulo[0], cx - q.w), uhi[0] = fmaxf(uhi[0], cx + q.w);
                ulo[1] = fminf(ulo[1], cy - q.w), uhi[1] = fmaxf(uhi[1], cy + q.w);
                ulo[2] = fminf(ulo[2], cz - q.w), uhi[2] = fmaxf(uhi[2], cz + q.w);
            }
        }
        const int lane = tid & 31, cw = ct >> 5, ncw = coll_threads >> 5;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                ulo[a] = fminf(ulo[a], __shfl_xor_sync(0xffffffffu, ulo[a], o));
                uhi[a] = fmaxf(uhi[a], __shfl_xor_sync(0xffffffffu, uhi[a], o));
            }
        }
        if (lane == 0)
#pragma unroll
            for (int a = 0; a < 3; ++a) s_ubox[cw][a] = ulo[a], s_ubox[cw][3 + a] = uhi[a];
        coll_sync();
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            ulo[a] = s_ubox[0][a], uhi[a] = s_ubox[0][3 + a];
            for (int w = 1; w < ncw; ++w) ulo[a] = fminf(ulo[a], s_ubox[w][a]), uhi[a] = fmaxf(uhi[a], s_ubox[w][3 + a]);
        }
        // candidate words: boxes 0-31, 32-63, obstacle spheres 0-31, 32-63
        for (int k0 = cw * 32; k0 < 4 * 32; k0 += coll_threads) {
            const int k = k0 + lane;
            bool near = false;
            if (k < 64) {
                if (k < pb.B) {
                    const float4 lo = s_boxlh[2 * k], hi = s_boxlh[2 * k + 1];
                    near = lo.x <= uhi[0] && hi.x >= ulo[0] && lo.y <= uhi[1] && hi.y >= ulo[1] && lo.z <= uhi[2] &&
                           hi.z >= ulo[2];
                }
            } else if (k - 64 < pb.O) {
                const float4 w = s_wsph[k - 64];
                const float ex = w.x - fminf(fmaxf(w.x, ulo[0]), uhi[0]);
                const float ey = w.y - fminf(fmaxf(w.y, ulo[1]), uhi[1]);
                const float ez = w.z - fminf(fmaxf(w.z, ulo[2]), uhi[2]);
                near = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= w.w * w.w;
            }
            const unsigned word = __ballot_sync(0xffffffffu, near);
            if (lane == 0) s_cand[k0 >> 5] = word;
        }
        coll_sync();
        const unsigned long long cb = s_cand[0] | (static_cast<unsigned long long>(s_cand[1]) << 32);
        const unsigned long long co = s_cand[2] | (static_cast<unsigned long long>(s_cand[3]) << 32);
        for (int idx = ct; idx < I * F; idx += coll_threads) {
            const float4 c = s_lcent[idx];
            unsigned long long mb = 0ull, mo = 0ull;
            for (unsigned long long m = cb; m; m &= m - 1ull) {
                const int b = __ffsll(static_cast<long long>(m)) - 1;
                const float4 lo = s_boxlh[2 * b], hi = s_boxlh[2 * b + 1];
                const float ex = c.x - fminf(fmaxf(c.x, lo.x), hi.x);
                const float ey = c.y - fminf(fmaxf(c.y, lo.y), hi.y);
                const float ez = c.z - fminf(fmaxf(c.z, lo.z), hi.z);
                if (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < c.w * c.w) mb |= 1ull << b;
            }
            for (unsigned long long m = co; m; m &= m - 1ull) {
                const int k = __ffsll(static_cast<long long>(m)) - 1;
                const float4 w = s_wsph[k];
                const float ex = c.x - w.x, ey = c.y - w.y, ez = c.z - w.z;
                const float rb = c.w + w.w;
                if (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < rb * rb) mo |= 1ull << k;
            }
            s_mask[2 * idx] = mb;
            s_mask[2 * idx + 1] = mo;
        }
        coll_sync();
    }

    // ---- sphere centres; world collision with its minimiser (sphere, obstacle);
    // each thread's (step, sphere) advances by coll_threads tasks without a division
    const int sph_dq = coll_threads / M, sph_dr = coll_threads - sph_dq * M;
    int sph_item = ct / M, sph_s = ct - sph_item * M;
    for (int idx = ct; idx < I * M; idx += coll_threads) {
        const int item = sph_item, s = sph_s;
        sph_item += sph_dq, sph_s += sph_dr;
        if (sph_s >= M) sph_s -= M, ++sph_item;
        const float4 q = s_sph[s];
        const float4* T = s_frame + item * FS + s_slink[s] * 3;
        const float4 r0 = T[0], r1 = T[1], r2 = T[2];
        float4 c;
        c.x = fmaf(r0.x, q.x, fmaf(r0.y, q.y, fmaf(r0.z, q.z, r0.w)));
        c.y = fmaf(r1.x, q.x, fmaf(r1.y, q.y, fmaf(r1.z, q.z, r1.w)));
        c.z = fmaf(r2.x, q.x, fmaf(r2.y, q.y, fmaf(r2.z, q.z, r2.w)));
        c.w = q.w;
        s_cent[idx] = c;
        float depth = 0.f;
        int best = -1;
        unsigned long long mb = all_b, mo = all_o;
        if (bp) {
            mb = s_mask[2 * (item * F + s_slink[s])];
            mo = s_mask[2 * (item * F + s_slink[s]) + 1];
        }
        while (mb) {  // ascending obstacle index, as the plain loop
            const int b = __ffsll(static_cast<long long>(mb)) - 1;
            mb &= mb - 1ull;
            const float4 lo = s_boxlh[2 * b], hi = s_boxlh[2 * b + 1];
            const float ex = c.x - fminf(fmaxf(c.x, lo.x), hi.x);
            const float ey = c.y - fminf(fmaxf(c.y, lo.y), hi.y);
            const float ez = c.z - fminf(fmaxf(c.z, lo.z), hi.z);
            if (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < c.w * c.w) {
                const float* bx = s_boxes + b * 6;
                const float qx = fabsf(c.x - bx[0]) - bx[3], qy = fabsf(c.y - bx[1]) - bx[4],
                            qz = fabsf(c.z - bx[2]) - bx[5];
                const float ox = fmaxf(qx, 0.f), oy = fmaxf(qy, 0.f), oz = fmaxf(qz, 0.f);
                const float sd = sqrtf(fmaf(ox, ox, fmaf(oy, oy, oz * oz))) +
                                 fminf(fmaxf(qx, fmaxf(qy, qz)), 0.f) - c.w;
                if (-sd > depth) {
                    depth = -sd;
                    best = b;
                }
            }
        }
        while (mo) {
            const int k = __ffsll(static_cast<long long>(mo)) - 1;
            mo &= mo - 1ull;
            const float4 w = s_wsph[k];
            const float ex = c.x - w.x, ey = c.y - w.y, ez = c.z - w.z;
            const float dist2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
            const float rs = c.w + w.w;
            if (dist2 < rs * rs && rs - sqrtf(dist2) > depth) {
                depth = rs - sqrtf(dist2);
                best = pb.B + k;
            }
        }
        if (best >= 0)
            atomicMax(s_keyw + item, depth_key(depth, static_cast<uint32_t>(s * NO + best)));
    }
    coll_sync();
    // ---- self collision with its minimiser: (step, pair block) tasks dealt
    // 32 at a time from a shared counter; the cost warp joins once its own work
    // is done (every task is taken once whoever takes it, and the minimiser is
    // an atomic max: the same result in any order)
    if (ct == 0) {  // (after the barrier that ended the world phase; release: the centres and bounds)
        __threadfence_block();
        *s_cflag = 1;
    }
    coll_self_tasks();
    for (int idx = ct; idx < I * pb.P; idx += coll_threads) {
        const int item = idx / pb.P, k = idx - item * pb.P;
        const uint32_t pr = s_pairs[k];
        const float4 ca = s_cent[item * M + (pr & 0xffff)], cb = s_cent[item * M + (pr >> 16)];
        const float ex = ca.x - cb.x, ey = ca.y - cb.y, ez = ca.z - cb.z;
        const float dist2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
        const float rs = ca.w + cb.w;
        if (dist2 < rs * rs)
            atomicMax(s_keys + item, depth_key(rs - sqrtf(dist2), static_cast<uint32_t>((1u << 24) + k)));
    }
    }  // the collision warps
    __syncthreads();

    // ---- collision gradients of each step's minimiser
    for (int h = tid; h < I; h += nt) {
        const float4* fr = s_frame + h * FS;
        float gth[kMaxDof];
#pragma unroll
        for (int k = 0; k < kMaxDof; ++k) gth[k] = (k < d) ? s_gth[h * d + k] : 0.f;
        float dworld = 0.f, dself = 0.f;
        const unsigned long long kw = s_keyw[h], ks = s_keys[h];
        if (kw) {
            dworld = __uint_as_float(static_cast<uint32_t>(kw >> 32));
            const uint32_t id = 0xffffffffu - static_cast<uint32_t>(kw & 0xffffffffu);
            const int s = id / NO, ob = id - s * NO;
            const float4 c = s_cent[h * M + s];
            float gx, gy, gz;
            if (ob < pb.B) {
                const float* bx = s_boxes + ob * 6;
                const float q[3] = {fabsf(c.x - bx[0]) - bx[3], fabsf(c.y - bx[1]) - bx[4],
                                    fabsf(c.z - bx[2]) - bx[5]};
                const float sg[3] = {c.x - bx[0] >= 0.f ? 1.f : -1.f, c.y - bx[1] >= 0.f ? 1.f : -1.f,
                                     c.z - bx[2] >= 0.f ? 1.f : -1.f};
                const float ox = fmaxf(q[0], 0.f), oy = fmaxf(q[1], 0.f), oz = fmaxf(q[2], 0.f);
                const float out = sqrtf(ox * ox + oy * oy + oz * oz);
                if (out > 0.f) {
                    gx = sg[0] * ox / out;
                    gy = sg[1] * oy / out;
                    gz = sg[2] * oz / out;
                } else {
                    const int km = (q[1] > q[0]) ? ((q[2] > q[1]) ? 2 : 1) : ((q[2] > q[0]) ? 2 : 0);
                    gx = km == 0 ? sg[0] : 0.f;
                    gy = km == 1 ? sg[1] : 0.f;
                    gz = km == 2 ? sg[2] : 0.f;
                }
            } else {
                const float4 w = s_wsph[ob - pb.B];
                const float ex = c.x - w.x, ey = c.y - w.y, ez = c.z - w.z;
                const float dist = sqrtf(ex * ex + ey * ey + ez * ez);
                const float inv = dist > 0.f ? 1.f / dist : 0.f;
                gx = ex * inv;
                gy = ey * inv;
                gz = ez * inv;
            }
            // c_world = -sd: d/dc = -grad sdf
            add_point_grad(fr, s_slink[s], c.x, c.y, c.z, -gx, -gy, -gz, pb.w_coll, gth);
        }
        if (ks) {
            dself = __uint_as_float(static_cast<uint32_t>(ks >> 32));
            const uint32_t id = 0xffffffffu - static_cast<uint32_t>(ks & 0xffffffffu);
            int a, b;
            if (id >= (1u << 24)) {
                const uint32_t pr = s_pairs[id - (1u << 24)];
                a = pr & 0xffff;
                b = pr >> 16;
            } else {
                const uint4 blk = s_pblk[id / kSelfBlockIds];
                const uint32_t r = id % kSelfBlockIds;
                a = blk.x + r / 8;
                b = blk.z + r % 8;
            }
            const float4 ca = s_cent[h * M + a], cb = s_cent[h * M + b];
            const float ex = ca.x - cb.x, ey = ca.y - cb.y, ez = ca.z - cb.z;
            const float dist = sqrtf(ex * ex + ey * ey + ez * ez);
            const float inv = dist > 0.f ? 1.f / dist : 0.f;
            const float nx = ex * inv, ny = ey * inv, nz = ez * inv;
            add_point_grad(fr, s_slink[a], ca.x, ca.y, ca.z, -nx, -ny, -nz, pb.w_coll, gth);
            add_point_grad(fr, s_slink[b], cb.x, cb.y, cb.z, nx, ny, nz, pb.w_coll, gth);
        }
        s_cost[h] += pb.w_coll * (dself + dworld);
#pragma unroll
        for (int k = 0; k < kMaxDof; ++k)
            if (k < d) s_gth[h * d + k] = gth[k];
    }
    __syncthreads();

    // ---- reverse scans (adjoint of Eq. 7) per joint; dC/du overwrites u
    for (int j = tid; j < d; j += nt) {
        float s1 = 0.f, s2 = 0.f;
        // (unrolled so that the loads of later steps issue ahead of the two
        // running sums, which keep their order)
#pragma unroll 6
        for (int h = H - 1; h >= 0; --h) {
            const float g = s_gpow[h];
            s1 = fmaf(g, s_gth[h * d + j], s1);
            const float tv = fmaf(s_dt[h], s1, g * s_gthd[h * d + j]);
            s2 += tv;
            float gu = g * s_gu[h * d + j];
            if (h + 1 < H) gu = fmaf(s_gpow[h + 1], s_gup[(h + 1) * d + j], gu);
            s_u[h * d + j] = fmaf(s_dt[h], s2, gu);
        }
    }
    __syncthreads();

    // ---- this particle's row: dC_n/du_n (none for null particles), C_n
    if (n >= pb.n_null)
        for (int o = tid; o < HD; o += nt) adj_add(acc.sum + o, s_u[o], kAdjGradScale, acc.bad);
    __shared__ int s_last;
    if (tid == 0) {
        float C = 0.f;
#pragma unroll 6
        for (int h = 0; h < H; ++h) C = fmaf(s_gpow[h], s_cost[h], C);
        if (Ctot) Ctot[n] = C;
        adj_add(acc.sum + HD, C, kAdjCostScale, acc.bad);
    }
    __syncthreads();  // every add of this CTA issued
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(acc.count, 1u) == static_cast<unsigned int>(pb.N - 1);
    }
    __syncthreads();
    if (!s_last) return;
    // ---- the last CTA: the sums are complete
    __threadfence();
    const bool bad = *reinterpret_cast<volatile int*>(acc.bad) != 0;
    const float invN = 1.f / static_cast<float>(pb.N);
    for (int o = tid; o <= HD; o += nt) {
        const long long v = static_cast<long long>(atomicExch(acc.sum + o, 0ull));  // read and clear
        const float tot = bad ? NAN
                              : static_cast<float>(static_cast<double>(v) / (o < HD ? kAdjGradScale : kAdjCostScale)) * invN;
        if (o < HD) {
            if (grad_out) grad_out[o] = tot;
            float m = pb.mu[o];
            if (eta != 0.f && !bad) {
                m -= eta * tot;
                pb.mu[o] = m;
            }
            if (finalize && o < d) cmd_out[o] = m;
        } else {
            if (J_out) *J_out = tot;
        }
    }
    if (tid == 0) {
        *acc.count = 0u;
        *acc.bad = 0;
        if (finalize) st->step += 1;
    }
}
