// Device-resident state of one bundle-adjustment problem and the launchers
// of every kernel of the hot path.
//
// Data layout in HBM (FP32 unless noted; k_j = observations of landmark j):
//   cams[9 n_cam], pts[3 n_pt]          current state; cand_* the candidate
//   obs_cam_s, obs_pt_s, obs_xy_s       observations sorted by (landmark, camera)
//   pt_off[n_pt + 1] (int32)            landmark j owns sorted obs pt_off[j] ..
//   cam_off[n_cam + 1], cam_list[n_obs] camera -> sorted positions (increasing)
//   a_off[n_pt + 1] (int64)             float offset of A_j in apool (blocks stored by
//                                       decreasing k: lm_by_k order)
//   apool                               A_j = Q^T J_p rows below R1, 2k x 9k row-major,
//                                       the last 3 rows are the landmark damping rows
//                                       (Sec. 5.3); blocks padded to 16 bytes
//   tpool                               top_j: 3 x (9k + 4) rows [Q1^T J_p | R1 | Q1^T r],
//                                       at float offset 3 (9 pt_off[j] + 4 j)
//   cpool                               c_j = Q2^T r (2k), at float offset c_off[j] (storage order)
//   rot[12 n_pt]                        six Givens (cos, sin) of the current damping
//   dp2[9 n_cam], dl2[3 n_pt]           D^2 = clamp(diag(J^T J), 1e-6, 1e32)
//   PCG vectors (9 n_cam each) and the per-camera 9x9 preconditioner blocks
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace sqrtba {

// Scalars of the PCG recursion, kept on the device so that a whole solve
// can run without host round trips.
struct PcgScalars {
    float rho;        // r^T z
    float q_prev;     // Q_{i-1} of the Nash-Sofer test
    float gnorm;      // ||g||
    float rnorm;      // ||r_i||
    float lambda;     // LM damping of the current blocks
    float eta;        // forcing tolerance
    int32_t it;       // iterations done
    int32_t max_it;
    int32_t done;     // 1 once a stop rule fired
    int32_t stop;     // reason (ba_pcg_report.stop_reason)
    int32_t warm;     // 1 if the learned warm start was kept
    int32_t pad;      // batch-wide scalars: iterations of the graph loop
};

// Levenberg-Marquardt state of one problem of a batch (device resident;
// the accept / reject decision runs on the device, Sec. 6.1 rules).
struct BatchLm {
    double lambda, nu;
    double cost;        // E at the current state
    double cost0;       // E at the initial state
    double new_cost;    // E at the last candidate
    double model_cost;  // L of the last step
    int32_t iter;       // linear solves done
    int32_t accepted;   // accepted steps
    int32_t cg_total;   // PCG iterations over all LM iterations
    int32_t stop;       // 0 running, 1 function tolerance, 2 iteration limit, 3 lambda limit
    int32_t active;     // 1 while the problem iterates
    int32_t finish;     // batch LM iteration after which the problem stopped (-1: running)
    int32_t last_acc;   // the last candidate was accepted
    int32_t pad;
};

// Work of a batch iteration per problem (null blm: a single problem, all work):
// a problem that has stopped does nothing; one whose last step was rejected
// keeps its linearisation (K1 skipped, K2 undoes and redoes its damping).
__device__ __forceinline__ bool batch_active(const BatchLm* blm, int b) { return !blm || blm[b].active; }
__device__ __forceinline__ bool batch_relin(const BatchLm* blm, int b) {
    return !blm || (blm[b].active && (blm[b].iter == 0 || blm[b].last_acc));
}

// Index spaces of a batch of independent problems concatenated into one
// problem (cameras, landmarks and observations of problem b are contiguous).
struct BatchState {
    int32_t n_prob = 0;                  // 0: a single problem
    int32_t *cam_prob = nullptr, *lm_prob = nullptr;  // owning problem of each camera / landmark
    int32_t *prob_cam_off = nullptr, *prob_lm_off = nullptr;  // [n_prob + 1]
    int64_t* prob_obs_off = nullptr;     // [n_prob + 1], sorted observation ranges
    float* lam = nullptr;                // [n_prob] damping of the current blocks
    PcgScalars* pcg = nullptr;           // [n_prob] per-problem CG scalars
    int32_t* n_done = nullptr;           // problems whose CG has stopped
    BatchLm* lm = nullptr;               // [n_prob]
    double *cost_a = nullptr, *cost_b = nullptr;  // [n_prob] segmented sums
    int32_t* n_active = nullptr;         // problems still iterating
    int32_t* n_active_host = nullptr;    // pinned mirror
    std::vector<int32_t> h_cam_off, h_lm_off;
    std::vector<int64_t> h_obs_off;
    std::vector<cudaEvent_t> iter_events;  // one per batch LM iteration (+ start)
    std::vector<int32_t> iter_active;      // problems iterating at the start of each batch LM iteration
    std::vector<float> iter_ms;            // duration of each batch LM iteration (events)
};

// Optional timing of the phases of the hot path with CUDA events.
enum ProfSlot { PROF_LINEARIZE = 0, PROF_DAMP, PROF_PRECOND, PROF_MATVEC, PROF_PCG_UPDATE,
                PROF_BACKSUB, PROF_COST, PROF_NSLOT };

struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> events;   // pairs handed out by begin()
    size_t next = 0;
    struct Pending {
        cudaEvent_t a, b;
        int slot;
    };
    std::vector<Pending> pending;
    double ms[8] = {};
    int64_t count[8] = {};
};

struct Problem {
    int32_t n_cam = 0, n_pt = 0;
    int64_t n_obs = 0;
    int32_t k_max = 0;
    int32_t n_big = 0;               // landmarks with k > 32 (CTA-per-landmark K1)
    int64_t sum_k2 = 0;
    int64_t a_floats = 0, t_floats = 0;
    ba_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t side = nullptr;     // second stream for work that overlaps (joined by events)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int sm_count = 0;

    // parameters
    float *cams = nullptr, *pts = nullptr, *cand_cams = nullptr, *cand_pts = nullptr;
    float *frames = nullptr, *cand_frames = nullptr;  // camera frames (R, t, f, k1, k2) of cams / cand_cams
    // sorted observations and index
    int32_t *obs_cam_s = nullptr, *obs_pt_s = nullptr, *perm = nullptr;
    float2* obs_xy_s = nullptr;
    int32_t *pt_off = nullptr, *cam_off = nullptr, *cam_list = nullptr;
    int64_t* a_off = nullptr;
    int32_t* lm_by_k = nullptr;      // landmarks by decreasing k (storage order of the blocks)
    int32_t* mv_cam = nullptr;       // camera of every observation in storage order
    int32_t* c_off = nullptr;        // float offset of c_j = Q2^T r (storage order, 2k per landmark)
    int32_t* cam_list_st = nullptr;  // camera lists as storage-order observation indices
    // chunks of at most PG_CHUNK observations of one camera (K3 in Gram form):
    // camera c owns chunks pg_chunk_off[c] .. pg_chunk_off[c + 1]
    int32_t *pg_chunk_off = nullptr, *pg_chunk_cam = nullptr;
    float* pg_part = nullptr;        // REC-sized partial sums per chunk
    int32_t pg_chunks = 0;
    std::vector<int32_t> k_run_count;  // host: landmarks with k = k_max - b
    std::vector<int64_t> run_off, run_co;  // host: float / observation offset of run b
    // work plans of the tile pipeline: tiles of the block pool streamed
    // through shared memory.  Blocks with k <= ksmall are grouped into tiles
    // of up to small_bytes; larger ones are cut into row tiles.  The matvec
    // (K4) and the preconditioner record pass (K3) have a plan each (the
    // autotuner chooses both).
    struct TilePlan {
        void* tiles = nullptr;           // MvTile[n]
        int32_t* begin = nullptr;        // first tile of each CTA (grid + 1)
        int n = 0, cap = 0;
        int ksmall = 21;
        int small_bytes = 32768;
        int64_t n_obs_split = 0;         // observations of blocks split into row tiles (first in storage order)
        int ns = 6;                      // pipeline depth (4, 5 or 6 stages)
        int y_smem = 1;                  // matvec: accumulate y in shared memory where it fits
        int big8_kmax = 40;              // matvec: row tiles with k up to this take 8 rows a warp (else 4)
    };
    TilePlan mv_plan, pc_plan;
    int mv_grid = 0;
    bool tuned = false;              // the autotuner has chosen the plan
    // blocks
    float *apool = nullptr, *tpool = nullptr, *cpool = nullptr, *rot = nullptr;
    // implicit storage (ba_options.implicit_blocks): per observation in storage
    // order 24 floats as 6 float4 chunks (chunk m of observation so at float4
    // index m n_obs + so): J_s rows (18) and Householder rows (6); residuals
    // (2 per observation, storage order); per storage position LM_REC floats
    // (the LR_* offsets below).  The top rows [Q1^T J_p | R1 | Q1^T r] are not
    // stored: camera s's 3 x 9 slice is D_s - P (V_s^T J_s), with D_s the
    // rows 0..2 of J_p in its columns (J_s itself for slot 0, J_s's first row
    // in row 2 for slot 1, zero otherwise) and P = V[0:3, :] Tm^T
    bool implicit = false;
    float *ipool = nullptr, *rpool = nullptr, *lmrec = nullptr;
    int32_t* lm_pos = nullptr;       // storage position of every landmark
    float* pq_part = nullptr;        // implicit storage: the matvec's per-CTA sums of ||A_j p||^2 (CG)
    int4* k3rec = nullptr;           // K3's camera-ordered records (landmark, storage index, position | slot)
    float2* k3xy = nullptr;          // and measurements, per camera-list entry
    float* init_part = nullptr;      // CG start folded into K3: per-camera partials of g^T g, r^T z
    uint32_t* init_ticket = nullptr; // and the finish kernel's completion count
    void* im_tasks = nullptr;        // matvec tasks (implicit.cu)
    int im_ntasks = 0;
    int im_nbig = 0;                 // matvec tasks with k > 32 (the first ones), handed out dynamically
    uint32_t* im_ctr = nullptr;      // their counter [0] and the CTAs-done count [32]
    // explicit Schur complement in FP32 (ba_options.schur_explicit, schur.cu):
    // block CSR of H~ with both triangles, pair -> blocks map, b~
    bool schur = false;
    int32_t *sc_row_ptr = nullptr, *sc_col = nullptr, *sc_diag_blk = nullptr, *sc_pair_blk = nullptr;
    int64_t* sc_pair_off = nullptr;
    int64_t sc_nblk = 0;
    float *sc_blk = nullptr, *sc_bt = nullptr;
    float *dp2 = nullptr, *dl2 = nullptr;
    // PCG
    float *g = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
    float *minv = nullptr, *mdiag = nullptr;
    float* prec = nullptr;           // 56 floats per observation: A_s^T A_s (upper), A_s^T c, 2 pad
    PcgScalars* pcg = nullptr;
    PcgScalars* pcg_host = nullptr;  // pinned mirror
    // step
    float* dl = nullptr;
    // reductions
    double* partials = nullptr;      // per-block FP64 partial sums
    double* dsum = nullptr;          // [0] cost, [1] model cost, [2] deferred cost; err follows at [4]
    double* dsum_host = nullptr;     // pinned mirror (6 doubles)
    uint32_t* err = nullptr;         // kernel error words (inside dsum's allocation, so that one copy
                                     // brings back the scalars and the errors): [0] ERRBIT_* bits,
                                     // [1] preconditioner blocks replaced by their diagonal,
                                     // [2] cameras whose Gram-form sums were replaced by sums over
                                     // the stored blocks (cancellation guard)
    uint32_t* err_host = nullptr;    // pinned mirror of err[0..3] (inside dsum_host); [3] receives
                                     // the attached model's error word
    int32_t precond_fallbacks = 0;   // err[1] at the last synchronisation
    int32_t precond_exact = 0;       // err[2] at the last synchronisation
    // failure test hooks of the matvec (ba_debug_fail_matvec): wait limit (0: WAIT_NS)
    // and a tile of CTA 0 that is never issued (-1: none)
    uint64_t dbg_wait_ns = 0;
    int32_t dbg_fail_tile = -1;
    int red_grid = 0;

    // CUDA graph of a chunk of PCG iterations
    cudaGraphExec_t pcg_graph = nullptr;
    int pcg_graph_iters = 0;
    int graph_kind = 0;              // 1 chunk of PCG_CHUNK iterations, 2 conditional WHILE loop
    bool pending_iteration_launches = false;  // WHILE launch: kernel count known after the sync
    bool capturing = false;
    std::vector<cudaEvent_t> mv_events;  // 2 per captured PCG iteration (profiling)

    // batch of independent problems (n_prob = 0 for a single problem)
    BatchState batch;

    // learned warm start and preconditioner correction (K8)
    struct Mlp* mlp = nullptr;       // attached model (not owned)
    float* lfeat = nullptr;          // [n_cam][19] features
    float* laux = nullptr;           // [n_cam][72] head inputs
    float* minv_l = nullptr;         // [n_cam][81] corrected block inverses B_i
    bool learned_active = false;     // the CG of this solve uses minv_l
    bool graph_learned = false;      // the captured graph was built with minv_l
    int64_t learned_fallbacks = 0;   // learned solves replaced by the plain CG

    // counters
    Profiler prof;
    int64_t launches = 0;      // kernels launched by the library
    int64_t h2d_bytes = 0, d2h_bytes = 0;

    // host-side LM state
    bool linearized = false, damped = false, solved = false, backsubbed = false;
    double lambda_damped = 0.0;
    double lambda = 1e-4, nu = 2.0;
    int32_t iteration = 0;
    bool stopped = false;
    double cost = 0.0;               // E at the current state
    bool cost_valid = false;         // cost holds E of the current state
    bool cost_pending = false;       // E of the current state is in dsum[2], not yet read back
    int64_t device_bytes = 0;
    std::vector<void*> allocations;
    std::string last_error;
};

// ---------------------------------------------------------------------------
// launchers (each enqueues on p.stream; none synchronises)
// ---------------------------------------------------------------------------
// K0: validation and grouping (index.cu)
void build_index(Problem& p, const int32_t* d_obs_cam, const int32_t* d_obs_pt,
                 const double* d_obs_xy, const double* d_cams, const double* d_pts);
// K1: damping diagonals, linearisation + Householder QR (linearize.cu)
void launch_frames(Problem& p);   // frames of the current cams
// K1 and D_p^2; cost_slot >= 0 adds the energy at the linearisation point
// (frames already computed) into dsum[cost_slot], run beside K1
void launch_linearize(Problem& p, int cost_slot = -1);
void launch_export_jacobians(Problem& p, float* r, float* jp, float* jl);
// cost and state update (cost.cu)
void launch_cost(Problem& p, bool candidate, int slot = 0);  // E into dsum[slot]
void launch_cost_on(Problem& p, const float* frames, const float* pts, int slot, cudaStream_t st);
void launch_candidate(Problem& p);
// K2: landmark damping with Givens rotations (damp.cu)
void launch_damp(Problem& p, bool undo_old, float lambda);
// K3, K5: preconditioner and PCG (pcg.cu); K4: matvec (matvec.cu)
// K3; with fuse_init (a single problem) the CG start is folded into its finish
// kernel: returns true if it was (no k_pcg_init needed)
bool launch_precond_rhs(Problem& p, bool fuse_init = false);
void build_k3_records(Problem& p);  // implicit storage: K3's camera-ordered records (at create)
void launch_pcg_init(Problem& p);
void launch_pcg_init_warm(Problem& p);
const float* active_minv(const Problem& p);
// in_while: the launch is captured into the body of a conditional WHILE
// graph node whose condition `cond` the update kernel clears when the CG stops
void launch_pcg_iteration(Problem& p, cudaEvent_t mv_begin = nullptr, cudaEvent_t mv_end = nullptr,
                          bool in_while = false, cudaGraphConditionalHandle cond = 0);
void launch_matvec(Problem& p, const float* v, float* y, bool add_damping);
void launch_matvec_raw(Problem& p, const float* v, float* y, const PcgScalars* S);
// implicit storage (implicit.cu): task plan, kernel attributes, y += A^T A v
void plan_implicit(Problem& p);
// explicit Schur complement (schur.cu): pattern from the sorted observations
// (host copies), D_l^2, assembly at lambda, preconditioner, matvec, back substitution
void plan_schur(Problem& p, const std::vector<int32_t>& pt_off, const std::vector<int32_t>& obs_cam_s);
void launch_schur_dl2(Problem& p);
void launch_schur_assemble(Problem& p, float lambda);
void launch_schur_precond(Problem& p);
void launch_schur_matvec(Problem& p, const float* v, float* y, const PcgScalars* S);
void launch_schur_backsub(Problem& p);
void launch_camera_diag(Problem& p);  // D_p^2 alone (linearize.cu)
void configure_implicit(Problem& p);
// pq_part (non-null): per-CTA sums of ||A_j v||^2, implicit_matvec_grid(p) of them
void launch_matvec_implicit(Problem& p, const float* v, float* y, const PcgScalars* S, float* pq_part = nullptr);
int implicit_matvec_grid(const Problem& p);
void launch_implicit_top_rows(Problem& p, int j, int k, float* top);  // export: landmark j's undamped top rows
void launch_precond_records(Problem& p);
int matvec_ctas_per_sm();
// K6: back substitution + model cost (backsub.cu)
void launch_backsub(Problem& p);
void launch_backsub_candidate_cost(Problem& p);
// batch: segmented FP64 sums, LM decision and commit (batch.cu)
void launch_batch_cost(Problem& p, bool candidate, double* out);
void launch_batch_start(Problem& p);
void launch_batch_decide(Problem& p, int iteration);
void launch_batch_commit(Problem& p);
// one-time kernel attributes (dynamic shared memory limits)
void configure_linearize(Problem& p);
void configure_matvec(Problem& p);
// tile plans (host planning + upload), after build_index: both plans, or
// one of them (pc = true: the preconditioner record pass's)
void plan_matvec(Problem& p);
void plan_tiles(Problem& p, bool pc);
// planner limits: largest mv_ksmall, largest mv_small_bytes
int matvec_ksmall_limit();
bool matvec_y_in_smem(const Problem& p);  // the matvec plan in use accumulates y in shared memory
int matvec_stage_bytes();

constexpr int PG_CHUNK = 256;  // observations per chunk of the Gram-form K3
// landmark record of the implicit storage (16-byte aligned groups)
constexpr int LM_REC = 64;     // floats per landmark
constexpr int LR_TM = 0;       // Tm, upper (00 01 02 11 12 22)                      K1
constexpr int LR_S = 6;        // S = G_dt^T G_dt, same order                          K2
constexpr int LR_GP = 12;      // G_tt P, row-major                                   K2
constexpr int LR_GT = 21;      // G_tt t (the damped Q1^T r)                          K2
constexpr int LR_G = 24;       // G_tt, row-major (undamped -> damped top rows)      K2
constexpr int LR_RD = 33;      // damped R, upper                                     K2
constexpr int LR_R1 = 40;      // undamped R1, upper                                  K1
constexpr int LR_DL2 = 46;     // D_l^2                                               K1
constexpr int LR_T = 49;       // t = Q1^T r (undamped)                               K1
constexpr int LR_P = 52;       // P = V[0:3, :] Tm^T, row-major                       K1

// kernel launch counter (not counted while a graph is being captured)
inline void count_launches(Problem& p, int n) {
    if (!p.capturing) p.launches += n;
}

// Device memory of every problem comes, in stream order, from one memory
// pool per device that keeps freed memory for the next problem (creating and
// destroying problems of similar size then maps no new memory); small pinned
// host buffers are recycled the same way.
cudaMemPool_t device_pool();
void* pinned_get(size_t bytes);
void pinned_put(void* ptr, size_t bytes);

// device allocation helper (stream-ordered on the problem's stream) that
// records the pointer for ba_destroy
template <typename T>
T* dalloc(Problem& p, int64_t n) {
    void* ptr = nullptr;
    size_t bytes = sizeof(T) * (size_t)(n > 0 ? n : 1);
    BA_CUDA_TRY(cudaMallocFromPoolAsync(&ptr, bytes, device_pool(), p.stream));
    p.allocations.push_back(ptr);
    p.device_bytes += (int64_t)bytes;
    return static_cast<T*>(ptr);
}

}  // namespace sqrtba
