// Internal state of an fmmbem_handle: geometry, octree, interaction lists,
// correction table and work buffers, all resident in device memory.
#pragma once
#include <vector>
#include "common.cuh"

struct fmmbem_handle {
    // problem
    int kernel = FMMBEM_LAPLACE;  // FMMBEM_LAPLACE or FMMBEM_STOKES
    int dof = 1;                  // unknowns per panel
    int ncomp = 1;                // harmonic expansions per cell and copy (1 Laplace, 4 Stokes, nrhs batched Laplace)
    int nrhs = 1;                 // vectors per mat-vec ([nrhs][N * dof] layout)
    // A batch of Stokes vectors keeps one copy of the expansion arrays per vector, copy r at
    // M + r esys (RHS-major): the tensor-core passes take every copy's rows in one launch, the
    // other kernels take the copy from blockIdx.y. 1 copy otherwise (a Laplace batch
    // interleaves its four vectors as components instead).
    int nsys = 1;
    size_t esys = 0;              // reals per copy: n_cells * ncomp * ESTRIDE
    int K = 4;                    // far-field Gauss points per panel
    int ncrit = 150;
    double theta = 0.5;
    fmmbem_opts opts{};
    int precision = FMMBEM_MIXED;
    int layer = FMMBEM_LAYER_SINGLE;  // operator of mat-vecs and solves (Laplace): V or 1/2 I + K
    cudaStream_t stream = nullptr;
    cudaStream_t stream2 = nullptr;  // near field runs here, concurrently with the far field
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // far-field pass before which a mat-vec releases its near field to the second stream
    // (0: P2M, 1: the first tree level, 2: M2L, 3: L2L); near_pending while not yet released.
    // After P2M: the first tensor-core tree level then finds SMs free, and the near-field blocks
    // fill the room its CTAs leave (headline 9.97 against 10.05 ms released before P2M); FP64
    // mat-vecs release it before P2M
    int near_at = 1;
    bool near_pending = false, near_fp64 = false;
    cudaStream_t istream = nullptr;  // internal stream of fmmbem_solve
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // one captured mat-vec per arithmetic and order p (input xfix, output kw), instantiated on
    // first use: slot p for the mixed arithmetic, FMMBEM_P_MAX + 1 + p for FP64 (the refined
    // solve alternates between them)
    static constexpr int NGRAPH = 2 * (FMMBEM_P_MAX + 1);
    bool use_graphs = true;
    cudaGraphExec_t mv_graph[NGRAPH] = {};
    int mv_graph_mode[NGRAPH] = {};
    int64_t graph_launches[NGRAPH] = {};
    int capturing = -1;          // slot of the graph being captured, else -1
    int pending_graph = -1;      // last replayed graph whose pass events await harvesting
    cudaEvent_t gev[NGRAPH][2 * FMMBEM_N_PASSES] = {};
    int gev_launches[NGRAPH][FMMBEM_N_PASSES] = {};
    int gev_tc[NGRAPH] = {};     // tc_pass_bits of each captured graph
    int tc_pass_bits = 0;               // passes of the mat-vec being issued that run on k_m2l_tc
    int64_t N = 0;   // panels
    int64_t NS = 0;  // Gauss points = K * N

    // geometry, in Morton-sorted panel order
    int* perm = nullptr;          // [N] sorted index -> caller's index
    int n_bodies = 1;
    int* body = nullptr;          // [N] body of each panel, sorted order (NULL: one body)
    double* body_acc = nullptr;   // [n_bodies][dof] sums of fmmbem_body_integrals
    double4* tgt_d = nullptr;     // [N] centroid (x,y,z, area)
    float4* tgt_f = nullptr;
    double4* nrm_d = nullptr;     // [N] unit normal (x,y,z, area)
    float4* nrm_f = nullptr;      // [N] the same in FP32 (mixed-precision double layer)
    float4* nrm_pt = nullptr;     // [N K] Stokes: each Gauss point's panel normal in FP32 (stresslet near field)
    double* verts = nullptr;      // [N][9] panel vertices
    double4* src_d = nullptr;     // [NS] Gauss point (x,y,z, q_k S_j), panel-major
    float4* src_f = nullptr;
    float4* src_rel = nullptr;    // [NS] Gauss point relative to its leaf centre, FP32 (x,y,z, q_k S_j)
    float4* tgt_rel = nullptr;    // [N] centroid relative to its leaf centre, FP32
    float4* src_w = nullptr;      // [NS] per mat-vec: leaf-relative position and weight q_k S_j x_j
    double origin[3] = {0, 0, 0};  // root-box centre; Stokes y.f strengths use it
    double half = 1.0;             // root-box half side
    double spill = 0.0;            // largest centroid-to-vertex distance

    // octree (cells in breadth-first order, levels contiguous)
    int n_cells = 0, n_leaves = 0, n_levels = 0;
    // shallowest level holding an M2L source / target: the multipoles of shallower cells are
    // never read and their local expansions stay zero, so M2M into and L2L out of the levels
    // above are skipped
    int m2m_lmin = 0, l2l_lmin = 0;
    std::vector<int> level_start;  // host, [n_levels + 1]
    double4* cell_cs = nullptr;    // [n_cells] centre (x,y,z) and side
    int2* cell_range = nullptr;    // [n_cells] sorted panel range [begin, end)
    double2* cell_rad = nullptr;   // [n_cells] cluster radii about the centre: (targets, Gauss points)
    int2* cell_child = nullptr;    // [n_cells] first child, number of children (0 = leaf)
    int* cell_level = nullptr;
    int* cell_parent = nullptr;
    int* leaves = nullptr;         // [n_leaves] cell ids
    int* parents = nullptr;        // non-leaf cells grouped by level (M2M and L2L blocks)
    std::vector<int> parent_start; // host, [n_levels + 1]: parents of level l are [parent_start[l], parent_start[l+1])
    int* leaf_class = nullptr;     // [n_leaves] leaves ordered by target count class (<=32, <=64, more)
    int leaf_class_start[4] = {0, 0, 0, 0};

    // interaction lists (CSR by target cell)
    int* m2l_ptr = nullptr;  // [n_cells + 1]
    int* m2l_src = nullptr;
    int64_t n_m2l = 0, n_m2l_same = 0;
    // M2L as batched products against precomputed operators (one per distinct pair geometry)
    bool m2l_tables = false;
    int* m2l_pt = nullptr;        // [n_m2l] target cell of each pair, grouped by operator
    int* m2l_ps = nullptr;        // [n_m2l] source cell
    int* m2l_refl = nullptr;      // [n_m2l] axis reflection mapping the pair's offset to its stored operator
    float* sign_f = nullptr;      // [8][ESTRIDE] coefficient signs of each reflection
    double* sign_d = nullptr;
    int4* m2l_tiles = nullptr;    // (operator, first pair, pair count, -)
    int n_tables = 0, n_tiles = 0, tab_ld = 0;
    size_t tab_stride = 0;
    double* tab_d = nullptr;      // [n_tables][2 ncoef(p_max)][tab_ld]
    float* tab_f = nullptr;
    // tensor-core (tcgen05) path: operators split into TF32 hi/lo, K-chunked core-matrix layout
    bool m2l_tc_ready = false;
    int m2l_mode = FMMBEM_M2L_TABLES;
    // per order p, mixed precision: M2L (m2l_tc_at) and M2M/L2L (tree_tc_at) on the tensor cores
    // (1) or on the SIMT kernels (0); set by fmmbem_set_tc_thresholds or fmmbem_autotune
    unsigned char m2l_tc_at[FMMBEM_P_MAX + 1] = {};
    unsigned char tree_tc_at[FMMBEM_P_MAX + 1] = {};
    float* tab_tc = nullptr;
    size_t tc_stride = 0;
    int tc_rows_max = 0;
    int tc_kc = 16;               // K width of the tensor-core operand chunks (tables and kernel)
    int4* m2l_tiles_tc = nullptr;
    int n_tiles_tc = 0;
    int* tc_src_info = nullptr;   // [n_tiles_tc][128]: source row offset * 8 + reflection (-1: empty row)
    int* tc_dst_info = nullptr;   // [n_tiles_tc][128]: target row offset * 8 + reflection
    int* tc_err = nullptr;        // set by the kernel if a bounded wait gives up
    // M2M / L2L on the tensor cores: one canonical operator each (TC layout), per-level tiles
    float* tree_tab_tc = nullptr;  // [2][tc_stride]: op 0 M2M, op 1 L2L
    int4* tree_tiles = nullptr;    // [2][n_tree_tiles]: operator index per tile (M2M tiles, then L2L tiles)
    int* tree_info = nullptr;      // [4][n_tree_tiles][128]: M2M src, M2M dst, L2L src, L2L dst row tables
    int n_tree_tiles = 0;
    std::vector<int> tree_tile_start;  // host, tiles of parent level l: [start[l], start[l+1])
    int n_sm = 152;
    int* kerr = nullptr;          // same, for the near-field bulk-copy kernel
    int* p2p_ptr = nullptr;  // [n_cells + 1]
    int* p2p_src = nullptr;
    int64_t n_p2p = 0, n_p2p_inter = 0;
    float4* p2p_rec = nullptr;  // [n_p2p] FP32 shift c_source - c_target (x,y,z) and first Gauss point (int bits)
    int* p2p_off = nullptr;     // [n_p2p] offset of the pair in its target leaf's source stream (self pair: empty)
    int* p2p_len = nullptr;     // [n_cells] length of each target leaf's source stream
    int* p2p_cnt = nullptr;     // [n_p2p] Gauss points of the source leaf
    int* p2p_toff = nullptr;    // [n_p2p] offset of the pair in its shared-memory stage
    int* stage_ptr = nullptr;   // [n_cells + 1] stages of each target leaf (bulk-copy P2P)
    int* stage_first = nullptr; // first pair of each stage
    int* stage_bytes = nullptr; // bytes of each stage
    int64_t n_stages = 0;
    int max_leaf_panels = 0;
    int4* p2p_items = nullptr;  // source-lane P2P work: (leaf, first target, target count), largest first
    int n_p2p_items = 0;
    int p2p_variant = 3;        // 0: shared stream tiles, 1: sliced L1 broadcast, 2: bulk-copied stages, 3: source lanes

    // near-singular / self corrections (CSR by sorted target panel), FP64
    int* corr_ptr = nullptr;   // [N + 1]
    int* corr_col = nullptr;
    double* corr_sl = nullptr;  // single layer: 1 (Laplace) or 9 (Stokes) per entry
    double* corr_dl = nullptr;  // double layer / stresslet
    float* corr_sl_f = nullptr;  // FP32 copies of both, read by the mixed-precision correction pass
    float* corr_dl_f = nullptr;
    int64_t n_corr = 0;

    // octant translation tables: R_n^m((+-1/4, +-1/4, +-1/4)) for the 8 children
    double* oct_d = nullptr;  // [8][NCOEF_MAX][2]
    float* oct_f = nullptr;

    // expansions: [n_cells][ncomp][NCOEF_MAX] complex, FP32 or FP64 view
    void* M = nullptr;
    void* L = nullptr;

    // mat-vec work, sorted order
    const double* xin = nullptr;  // input of the mat-vec in flight (sorted order)
    double* xs = nullptr;     // [N*dof]
    double* ys = nullptr;     // [N*dof]
    double* ynear = nullptr;  // [N*dof]
    double* ycorr = nullptr;  // [N*dof]: the correction rows' products of the work-item near field

    // Krylov work
    int kr_m = 0;
    double* V = nullptr;        // [(m+1) * n]
    double* kw = nullptr;       // [n]
    double* xfix = nullptr;     // [n] input of the captured mat-vecs
    double* kb = nullptr;       // [n] sorted rhs
    double* kx = nullptr;       // [n] sorted solution
    double* kr = nullptr;       // [n] residual
    double* kpart = nullptr;    // partial dots
    double* kh = nullptr;       // [m+2] dot results
    double* kh_host = nullptr;  // pinned
    double* kyv = nullptr;      // [m] update coefficients
    double* rf_r = nullptr;     // [n] outer residual of the refined solve (FMMBEM_MIXED_REFINED)
    double* rf_d = nullptr;     // [n] its inner correction
    // fused Arnoldi step (cooperative launch)
    int arn_blocks = 0;
    unsigned* arn_bar = nullptr;       // grid barrier counter and generation
    unsigned wait_limit = 1u << 26;    // polls before a grid-barrier wait gives up (fmmbem_set_wait_limit)
    double* arn_out_host = nullptr;    // mapped pinned: h1[65], h2[65], ||w||^2
    double* arn_out_dev = nullptr;

    // timing
    double setup_seconds = 0.0;
    bool prof_on = false;
    bool prof_serial = false;  // profiled mat-vecs run the near field on the far field's stream
    fmmbem_profile prof{};
    cudaEvent_t ev[2 * FMMBEM_N_PASSES] = {};
    void* prof_state = nullptr;  // per-handle event pool and pending intervals (capi.cu)
    int64_t launches = 0;
    // device-resident GMRES cycle (fmmbem_set_device_loop): one graph per restart cycle whose
    // while node repeats mat-vec (a switch over the orders) -> Arnoldi step -> Givens step on
    // the device until the cycle ends; built on first use for the handle's kernel selection
    bool dloop_on = false;
    cudaGraphExec_t dloop_exec = nullptr;
    uint64_t dloop_key = 0;
    void* dloop_state = nullptr;       // device cycle state
    void* dloop_host = nullptr;        // pinned copy read back after each cycle
    double* dloop_out = nullptr;       // the Arnoldi step's output (device)
    int64_t dloop_mv_launches[FMMBEM_P_MAX + 1] = {};
};

namespace fmmbem {
// setup.cu
int build_geometry_tree_lists(fmmbem_handle* h, const fmmbem_mesh* mesh);
// m2l.cu
int build_m2l_tables(fmmbem_handle* h);
int m2l_gemm(fmmbem_handle* h, int p, bool fp64);
// m2l_tc.cu
int build_m2l_tc(fmmbem_handle* h);
int m2l_tc(fmmbem_handle* h, int p);
int tree_tc(fmmbem_handle* h, int p, int level, int which);
int tree_tc_zero(fmmbem_handle* h, int p);
int m2l_tc_zero(fmmbem_handle* h);  // zero the local expansions the tensor-core M2L accumulates into
// fmm.cu
int far_field(fmmbem_handle* h, int p, bool fp64);
int far_eval_add(fmmbem_handle* h, int p, bool fp64, double* y_sorted, double scale);
int expansion_eval(int kind, int p, const double* center, double scale, int n_src, const double* src,
                   int n_tgt, const double* tgt, double* out, cudaStream_t st);
int init_octant_tables(fmmbem_handle* h);
// near.cu
int init_near_attrs();
int pack_sources(fmmbem_handle* h);
int near_field(fmmbem_handle* h, bool fp64, cudaStream_t st);
int near_release(fmmbem_handle* h, int stage);
int direct_field(fmmbem_handle* h, bool fp64, int which, const double* x_sorted, double* y_sorted);
// krylov.cu
int relaxed_p(double eta, double rho_prev, int p_initial, int p_min);
int arnoldi_blocks();
int gmres_solve(fmmbem_handle* h, const double* b_sorted, double tol, int relax, int p_initial, int p_min,
                double* x_sorted, int* iters, int* p_hist, double* res_hist, double* true_res);
int read_wait_flags(fmmbem_handle* h, cudaStream_t st);
// peaks.cu
int peak_rate(int kind, int blocks, int64_t iters, double* ops, double* ms, cudaStream_t st);
// sort.cu: stable LSD radix sorts of keys [0, end_bit) (values optional: NULL), and prefix sums;
// outputs must not alias inputs except for the scans; temporaries are stream-ordered on st
int radix_sort(const uint64_t* kin, uint64_t* kout, const int* vin, int* vout, int64_t n, int end_bit, cudaStream_t st);
int radix_sort(const uint32_t* kin, uint32_t* kout, const int* vin, int* vout, int64_t n, int end_bit, cudaStream_t st);
int exclusive_scan(const int* in, int* out, int64_t n, cudaStream_t st);
int inclusive_scan(const int* in, int* out, int64_t n, cudaStream_t st);
// capi.cu
int matvec_sorted(fmmbem_handle* h, int p, const double* xs, double* ys);
int matvec_capture_body(fmmbem_handle* h, int p);  // the mat-vec xfix -> kw at order p onto h->stream
uint64_t matvec_modes_key(const fmmbem_handle* h);  // kernel selection of every order's mat-vec
void dloop_free(fmmbem_handle* h);
void prof_begin(fmmbem_handle* h, int pass);
void prof_end(fmmbem_handle* h, int pass, int launches);
void prof_harvest(fmmbem_handle* h);
}  // namespace fmmbem
