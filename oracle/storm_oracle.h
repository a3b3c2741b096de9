/*
 * storm_oracle.h -- FP64 CPU oracle for one STORM sampling-based MPC control step.
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA path; only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no code, header, table or constant generator with the CUDA
 * library, and the CUDA library never calls it.
 *
 * Every routine is a plain, sequential restatement of the method of Bhardwaj et
 * al., "STORM: An Integrated Framework for Fast Joint-Space Model-Predictive
 * Control for Reactive Manipulation" (arXiv 2104.13542), in double precision.
 * Each function cites the section / equation / algorithm it follows.  Where the
 * paper is silent or garbled, the reading taken is stated next to the routine.
 *
 * Layouts (row-major, C order):
 *   dh          d x 4   (a_{i-1}, alpha_{i-1}, d_i, theta_offset_i), modified DH (Craig)
 *   sphere      M x 4   (x, y, z in the frame of its link, radius)
 *   sphere_link M       frame index 0..d the sphere is rigidly attached to
 *   pairs       P x 2   sphere indices checked for self-collision
 *   boxes       B x 6   (cx, cy, cz, hx, hy, hz) axis-aligned boxes
 *   wspheres    S x 4   (cx, cy, cz, r) obstacle spheres
 *   mu          H x d   mean control sequence (joint accelerations)
 *   sigma       d       per-joint standard deviation
 *   eps         N x S x d  standard-normal noise (S = knots, or H when no spline)
 *   u           N x H x d  sampled controls
 *   goal        7       (x, y, z, qw, qx, qy, qz)
 *   state       3 x d   (theta, theta_dot, theta_ddot)
 */
#ifndef STORM_ORACLE_H
#define STORM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_SAMPLER_PHILOX = 0, ORC_SAMPLER_HALTON = 1 };
enum { ORC_ROT_QUAT = 0, ORC_ROT_FROBENIUS = 1 };
enum { ORC_FILTER_DEFAULT = 0, ORC_FILTER_COMB = 1, ORC_FILTER_MIXED = 2 };
/* pos, rot, stop, joint, manip, self, world, smooth, ee speed, ee acceleration, ball */
enum { ORC_NTERMS = 11 };

typedef struct {
    int dof;
    const double* dh;
    const double* q_min;
    const double* q_max;
    int n_spheres;
    const int* sphere_link;
    const double* sphere;
    int n_pairs;
    const int* pairs;
} orc_robot;

typedef struct {
    int n_boxes;
    const double* boxes;
    int n_spheres;
    const double* spheres;
} orc_world;

typedef struct {
    int N, H, K;
    int n_knots;            /* 0: no smoothing, noise drawn per horizon step */
    int sampler;            /* ORC_SAMPLER_* */
    int n_null;             /* particles 0..n_null-1 are zero-acceleration particles */
    const double* dt;       /* H */
    double beta, gamma, alpha_mu, alpha_sigma, sigma_min;
    double w_pos, w_rot, w_stop, w_joint, w_manip, w_coll, w_smooth;
    double pos_axis_w[3];   /* alpha_2 of Eq. 9 */
    double rot_axis_w[3];   /* alpha_1 of Eq. 9 (Frobenius mode only) */
    int rot_mode;           /* ORC_ROT_* */
    double k_jl, k_m, qdd_max;
    uint64_t seed;
    uint32_t instance;
    int grad_steps;         /* gradient refinement steps after the K iterations */
    double grad_eta;        /* mu <- mu - grad_eta dJ/dmu */
    /* smoothing of the sampled noise along the horizon (Sec. 4.3):
     *   DEFAULT  B-spline through n_knots samples when n_knots > 0, else none;
     *   COMB     comb filter with coefficients comb[0..2] on H samples;
     *   MIXED    H samples per particle; the first round(mix_bspline (N - n_null))
     *            non-null particles take the B-spline through their first n_knots
     *            samples, the others the comb filter */
    int filter;
    double comb[3];
    double mix_bspline;
    /* task-space limits on the end-effector linear speed |v| and acceleration |a|
     * of Eq. 8's X_dot and X_ddot (terms added to the paper's list) */
    double w_ee_vel, w_ee_acc, ee_vel_max, ee_acc_max;
    /* ball on a tray held by the end effector (appendix, ball balancing) */
    double w_ball;
    double gravity[3];      /* g in the world frame */
    double tray_center[3];  /* tray centre in the end-effector frame */
    const double* ball;     /* 6: ball position, velocity (world) at the current state; NULL: none */
    int halton_scramble;    /* Halton sampler: linearly scrambled digits (multipliers from the seed) */
    /* learned self-collision network (Sec. 4.2, Eq. 13), evaluated per (particle, step)
     * by orc_mlp_arch_forward with its BF16 rounding points:
     *   mlp_mode 0  the exact sphere check (default);
     *            1  gate: the exact check only where the prediction (distance, positive
     *               apart) is below mlp_margin, elsewhere the self term is 0;
     *            2  cost: the self term is max(0, prediction), the network predicting the
     *               penetration depth (positive when colliding), no exact check */
    int mlp_mode;
    const double* mlp_params;          /* flat parameters, orc_mlp_arch layout */
    int mlp_enc, mlp_h1, mlp_h2, mlp_h3; /* its architecture (see orc_mlp_arch) */
    double mlp_margin;
} orc_params;

/* ---- noise ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform_from_bits(uint32_t x);
void orc_box_muller(double u1, double u2, double* z0, double* z1);
void orc_noise_philox(uint64_t seed, uint32_t step, uint32_t instance, uint32_t iter,
                      uint32_t tag, long long count, double* eps);
double orc_radical_inverse(uint64_t i, int base);
int orc_nth_prime(int n);
double orc_norm_ppf(double p);
void orc_noise_halton(int N, int S, int d, double* eps);
double orc_radical_inverse_scrambled(uint64_t i, int base, int mult);
int orc_halton_multiplier(uint64_t seed, int dim, int base);
void orc_noise_halton_ex(int N, int S, int d, int scramble, uint64_t seed, double* eps);
void orc_bspline_basis(int H, int S, double* B);

/* ---- rollout stages ---- */
void orc_smooth_controls(const orc_params* P, int d, const double* mu, const double* sigma,
                         const double* eps, double* u);
void orc_integrate(int H, int d, const double* dt, const double* state, const double* u,
                   double* theta, double* theta_dot);
void orc_fk(const orc_robot* R, const double* theta, double* frames);
void orc_jacobian(const orc_robot* R, const double* frames, double* J);
double orc_det(int n, const double* A);
double orc_manipulability(const double* J, int d);
void orc_quat_from_rot(const double* Rm, double* q);
void orc_rot_from_quat(const double* q, double* Rm);
double orc_box_sdf(const double* p, const double* box);
double orc_self_min_sd(const orc_robot* R, const double* frames);
double orc_world_min_sd(const orc_robot* R, const orc_world* W, const double* frames);
void orc_comb_filter(int H, int d, const double* c, const double* eps, double* out);
void orc_ee_twist(const orc_robot* R, const double* frames, const double* theta_dot,
                  const double* theta_ddot, double* xd, double* xdd);
int orc_ball_states(const orc_robot* R, const orc_params* P, const double* state,
                    const double* theta, double* x_ball, double* v_ball);
void orc_running_cost(const orc_robot* R, const orc_world* W, const orc_params* P,
                      const double* goal, int h, const double* theta_h,
                      const double* theta_dot_h, const double* u_h, const double* u_prev,
                      double* terms, double* total);
/* Threads of orc_rollout's loop over particles (default 1; results are the
 * same bits for every count). */
void orc_set_threads(int n);
int orc_get_threads(void);
int orc_rollout(const orc_robot* R, const orc_world* W, const orc_params* P,
                const double* state, const double* goal, const double* mu,
                const double* sigma, const double* eps, double* u, double* theta,
                double* theta_dot, double* ee, double* terms, double* cost, double* Ctot);
int orc_update(const orc_params* P, int d, const double* Ctot, const double* u,
               double* mu, double* sigma, double* weights);
void orc_shift(int H, int d, double* mu);
void orc_running_cost_grad(const orc_robot* R, const orc_world* W, const orc_params* P,
                           const double* goal, int h, const double* theta_h,
                           const double* theta_dot_h, const double* u_h, const double* u_prev,
                           double* g_theta, double* g_theta_dot, double* g_u, double* g_u_prev);
void orc_integrate_adjoint(int H, int d, const double* dt, const double* g_theta,
                           const double* g_theta_dot, const double* g_u, double* dC_du);
int orc_cost_grad(const orc_robot* R, const orc_world* W, const orc_params* P,
                  const double* state, const double* goal, const double* mu, const double* sigma,
                  const double* eps, double* grad_mu, double* J, double* dC_du);
/* ---- self-collision surrogate network (parameters flat, see storm_oracle.c) */
enum { ORC_MLP_IN = 16, ORC_MLP_HID = 256 };
enum { ORC_ENC_SCALED = 0, ORC_ENC_SINCOS = 1 };
typedef struct {
    int enc;           /* ORC_ENC_* */
    int h1, h2, h3;    /* hidden widths (each <= 256) */
} orc_mlp_arch;
long orc_mlp_arch_param_count(const orc_mlp_arch* A);
void orc_mlp_arch_encode(const orc_mlp_arch* A, const double* theta, int dof, double* x);
void orc_mlp_arch_forward(const orc_mlp_arch* A, const double* params, const double* theta, int B, int dof,
                          int bf16, double* y);
double orc_mlp_arch_loss_grad(const orc_mlp_arch* A, const double* params, const double* theta,
                              const double* target, int B, int dof, int bf16, double* grad);
long orc_mlp_param_count(void);
float orc_bf16_round(float x);
void orc_mlp_encode(const double* theta, int dof, double* x);
void orc_mlp_forward(const double* params, const double* theta, int B, int dof, int bf16,
                     double* y);
double orc_mlp_loss_grad(const double* params, const double* theta, const double* target, int B,
                         int dof, int bf16, double* grad);
double orc_self_min_sd_theta(const orc_robot* R, const double* theta);
int orc_step(const orc_robot* R, const orc_world* W, const orc_params* P,
             const double* state, const double* goal, uint32_t step, double* mu,
             double* sigma, double* cmd, double* best_cost);

#ifdef __cplusplus
}
#endif
#endif
