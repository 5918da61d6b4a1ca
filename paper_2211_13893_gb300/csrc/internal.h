// Internal declarations of libmsgfem (not part of the C ABI).
//
// Layouts (FP64):
//  * Omega*_j is a node box [I0, I1] x [J0, J1] x [0, NZ]; in-layer node
//    q = (i - I0) * nyn + (j - J0); local node n = k * npl + q; full-layout
//    row 3 n + c.  A "multivector" is [nfull][PST] row-major (PST columns).
//  * Layer blocks: for M in {K, A11} the DoFs of one node layer kept by M are
//    numbered compactly (c = 0 .. nM - 1) and padded with identity rows to bM
//    (a multiple of TILE).  Diagonal blocks D_l and sub-diagonal blocks E_l
//    (rows layer l + 1, columns layer l) are stored contiguously, bM x bM
//    row-major; after factorisation D_l holds L_l, E_l holds L_{l+1,l} and
//    a separate array holds Linv_l = L_l^{-1}.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "msgfem.h"

#define TILE 64
#define PST 32
#define KB 8      // block width of the block Krylov eigensolver
#define MQ 96     // largest Krylov basis (12 blocks)

// Tile task: C(64x64) = [C +] sign * [P *] A(64 x K) * op(B), or with
// G_POTRF the Cholesky factor and inverse of the SPD tile C (in place) with the
// inverse written to P.
// G_TRIB: B is a lower-triangular 64 x 64 tile (a diagonal block inverse) and
// K = 64; the FP64 tile kernel skips its all-zero 16 x 16 blocks.  G_SYMC: C is
// a diagonal tile whose upper triangle is never read (a Cholesky update); the
// FP64 tile kernel forms only its 16 x 16 blocks on or below the diagonal
enum { G_TRANSB = 1, G_ACC = 2, G_NEG = 4, G_POSTMUL = 8, G_POTRF = 16, G_TRIB = 32, G_SYMC = 64 };
template <typename T>
struct TileTaskT {
  const T* A;
  const T* B;
  T* C;
  const T* P;   // G_POSTMUL: 64x64 tile with leading dimension ldc; G_POTRF: inverse output
  int lda, ldb, ldc, K;
  int flags, sub;
};
using GemmTask = TileTaskT<double>;


// Solve step: C(64 x PST) = init + sign * op(A) * B
enum { S_TRANSA = 1, S_NEG = 2, S_INIT_GATHER = 4, S_INIT_TILE = 8, S_SCATTER = 16 };
template <typename T>
struct SolveTaskT {
  const T* A;
  const T* B;           // K x PC compact
  T* C;                 // 64 x PC compact tile
  const T* init;        // S_INIT_TILE: 64 x PC compact tile
  const int* gmap;      // S_INIT_GATHER: 64 in-layer full rows (or -1)
  const int* smap;      // S_SCATTER: 64 in-layer full rows (or -1)
  int lda, K, flags, sub, row_off;
};
using SolveTask = SolveTaskT<double>;

// multivector selectors
enum { MV_PHI = 0, MV_Z, MV_KPHI, MV_W, MV_T1, MV_R, MV_BR, MV_EV, MV_CB, MV_CW,
       MV_QB, MV_ZB, MV_WB, MV_TB, MV_NQ,
       MV_P1, MV_P2, MV_P3 };   // QB, NQ: [nfull][MQ]; ZB, WB, TB, P1-P3: [nfull][KB]
enum { GM_G1 = 0, GM_G2, GM_G3, GM_Y };

// Device-visible per-subdomain descriptor.
struct SubDev {
  int inst;                    // instance of the batch this subdomain belongs to
  int I0, I1, J0, J1;          // Omega* node box
  int oI0, oI1, oJ0, oJ1;      // Omega node box
  int nxn, nyn, nzn, npl, nnode, nfull;
  int nK, nA, bK, bA;          // compact / padded layer sizes
  int floating;
  int pin[6];                  // pinned full-layout rows (floating), -1 unused
  int loaded;                  // Omega* touches the loaded face x = L
  double* stencil;             // [nnode][27][9]
  double* mu;                  // [nnode]
  const signed char* cls;      // [npl] 1, 2, 3
  int* mapK; int* mapA;        // [bK], [bA]
  int* invK; int* invA;        // [3 npl]
  double* DK; double* EK; double* LK;   // [nzn][bK^2], [nzn-1][bK^2] (contiguous after DK), [nzn][bK^2]
  double* DA; double* EA; double* LA;
  double* ycK; double* ycA;    // [nzn][b][PST]
  double* rcK; double* rcA;    // [b][PST]
  double* Phi; double* Z; double* KPhi; double* W; double* T1;
  double* R; double* BR; double* EV; double* CB; double* CW;   // [nfull][PST]
  double* bload;               // [nfull]
  double* psi;                 // [nfull]
  double* G1; double* G2; double* G3; double* Y;   // [PST][PST]
  double* theta;               // [PST]
  double* resid;               // [PST]
  int* status;                 // [4]: 1 RR pencil degenerate, 2 kept basis columns
  // block Krylov eigensolver
  double* QB;                  // [nfull][MQ] N-orthonormal basis (A-harmonic vectors)
  double* NQ;                  // [nfull][MQ] N QB, kept with the basis (no stencil to re-form it)
  double* Zb; double* Wb; double* Tb;   // [nfull][KB] working blocks
  double* P1; double* P2; double* P3;   // [nfull][KB] preconditioned CG of the mixed K solves: z, p, q
  double* ycK8; double* ycA8;  // [nzn][b][KB] compact solve buffers
  double* rcK8; double* rcA8;  // [b][KB]
  // FP32 copies for the mixed-precision path (layer blocks, factors, solve buffers)
  float* DKf; float* EKf; float* LKf;
  float* DAf; float* EAf; float* LAf;
  float* ycK8f; float* ycA8f; float* rcK8f; float* rcA8f;   // KB columns
  float* ycKf; float* ycAf; float* rcKf; float* rcAf;       // PST columns
  double* H;                   // [MQ + KB][MQ] projected operator Q^T T M Q and R_{m+1}
  double* Hc;                  // [MQ][KB] block inner products
  double* Yk;                  // [MQ][PST] Ritz coefficients of the wanted pairs
};

// A schedule is a set of independent groups (each a sequence of steps, run on
// its own stream); steps[g] lists the launches of group g in order.
#define NGROUP 32   // most stream groups a schedule may use (16 by default; the autotuner may take 32)
struct SchedStep { int first, count; };
template <typename T>
struct ScheduleT {
  using Step = SchedStep;
  std::vector<std::vector<Step>> steps;
  std::vector<TileTaskT<T>> gemm;
  TileTaskT<T>* d_gemm = nullptr;
  bool k32 = true;   // every GEMM task's inner dimension is a multiple of 32
};
using Schedule = ScheduleT<double>;

template <typename T>
struct SolveScheduleT {
  using Step = SchedStep;
  std::vector<std::vector<Step>> steps;
  std::vector<SolveTaskT<T>> tasks;
  SolveTaskT<T>* d_tasks = nullptr;
  int kmax = 0;   // largest inner dimension of a task (shared-memory sizing)
  bool k64 = true;   // every inner dimension is a multiple of 64
};
using SolveSchedule = SolveScheduleT<double>;

// Fork/join of the group streams around a schedule run.
struct StreamSet {
  cudaStream_t s[NGROUP] = {};
  cudaEvent_t fork = nullptr, join[NGROUP] = {};
};

// Static schedules of one wave of subdomains (FP64, or FP32 in mixed precision).
struct WaveSched {
  std::vector<int> members;          // subdomains of the wave
  ScheduleT<double> fact;
  SolveScheduleT<double> solveK, solveA;     // PST columns
  SolveScheduleT<double> solveK8, solveA8;   // KB columns
  ScheduleT<float> factf;                    // mixed precision: FP32 factorisation
  SolveScheduleT<float> solveKf, solveAf, solveK8f, solveA8f;
  // persistent FP32 factorisation: per task in ticket order (counter of its
  // step, counter of the previous step or -1, tasks in that step, index in factf)
  std::vector<int4> pmeta;
  int pcount = 0;                            // step counters
  int4* d_pmeta = nullptr;
  int* d_pcount = nullptr;                   // pcount counters, then the ticket
};
// Ticket order and step dependencies of a factorisation schedule for the
// persistent kernel: a list schedule on `workers` resident CTAs (setup.cpp)
void build_persistent_meta(const ScheduleT<float>& s, std::vector<int4>& meta, int& pcount, int workers);

struct CoarsePair { int s, t, x0, x1, y0, y1; };   // (i, j) node box of Omega_s cap Omega*_t

// Host copies of the per-subdomain set-up arrays (uploaded once).
struct HostSub {
  std::vector<signed char> cls;
  std::vector<int> mapK, mapA, invK, invA;
  std::vector<double> mu, bload;
};

// A start block registered for the block Krylov eigensolver (learned warm start).
struct WarmStart {
  const float* X0 = nullptr;   // device [n2][ld], first ncols columns used
  int ld = 0, ncols = 0;
};

struct msgfem {
  int NX = 0, NY = 0, NZ = 0;
  double hx = 0, hy = 0, hz = 0, traction = 0;
  std::vector<double> h_xyz;         // node coordinates (general mesh), empty for the box
  std::vector<double> h_frame;       // per-element ply frames, empty = x, y, z
  std::vector<double> h_load;        // nodal loads [n_nodes][3], empty = the end-face traction
  std::vector<int> boxes;            // explicit non-overlapping element boxes, 4 per subdomain
  double* d_xyz = nullptr;           // device copies (nullptr for the box / default frames)
  double* d_frame = nullptr;
  double E9[9];
  int sx = 0, sy = 0, o = 0, os = 0;
  msgfem_options opt;
  cudaStream_t stream = nullptr;
  StreamSet gs;                      // streams of independent schedule groups
  cudaStream_t cap = nullptr;        // private stream on which schedules are captured as graphs
  std::map<uint64_t, std::pair<cudaGraphExec_t, long long>> graphs;   // key -> (graph, kernel nodes)
  int ngroup = NGROUP;               // groups in use (msgfem_options.streams, or the autotuner's choice)
  int ngroup_created = NGROUP;       // streams created at set-up
  int solve_variant = 0;             // kernel of the KB-wide block solves (SOLVE_*)
  int factor_left = 0;               // factorisation schedule: 0 right-looking, 1 left-looking
  int ngroup_factor = NGROUP;        // stream groups of the factorisation schedules
  int N = 0;
  int S = 1;                         // instances of the mesh batched in this handle
  int N0 = 0;                        // subdomains per instance (N = S N0)
  int layered = 0, ntypes = 0, type_cap = 0;
  int typed = 0;                     // curved mesh: element -> type map in d_etype
  int* d_etype = nullptr;            // [S nel] type of every element (typed)
  int* d_trep = nullptr;             // [ntypes] first element of every type (typed)
  int trep_cap = 0;
  std::vector<double> h_angles;
  std::vector<SubDev> sub;
  std::vector<HostSub> hsub;
  std::vector<int> n1, n2, n3, iters, basis_m, m_final;
  std::vector<int> krylov_left;      // [N] 1 if the last block Krylov run left the subdomain unconverged
  std::vector<int> cold_restart;     // [N] 1 if a registered start block was dropped for a cold start
  std::vector<double> lam_host;      // [N][n_loc] eigenvalues of the last local stage (rigid zeros first,
                                     // NaN from a subdomain's own count nloc_j on)
  std::vector<int> nloc_j;           // [N] eigenpairs of every subdomain in the last local stage
  std::vector<int> m_sel;            // [N] eigenvectors in the coarse basis (threshold selection)
  std::vector<int> thr_reached;      // [N] 0 if all n_loc eigenvalues were below the threshold
  std::vector<int> act_host;         // host copy of the active flags last uploaded
  std::vector<int> base_act;         // members of the wave being processed (all ones: one wave)
  std::vector<double> resid_max;
  std::vector<std::pair<void*, size_t>> allocs;   // device blocks of the handle and their sizes
  SubDev* d_sub = nullptr;
  double* d_E9 = nullptr;
  double* d_angles_type = nullptr;   // [ntypes]
  double* d_Ke = nullptr;            // [ntypes][576]
  double* d_gram_part = nullptr;
  int* d_flags = nullptr;            // [N + 1] active flags (entry N: coarse, always 1)
  int* d_flags_saved = nullptr;      // [N + 1] flags saved around an adaptive refinement
  double* d_rprev = nullptr;         // [N][KB] residual norms of the previous refinement step
  double* d_rref = nullptr;          // [N][KB] reference residual norms of the refinement
  double* d_pcg = nullptr;           // [N][4][KB] CG scalars per column: r.z, p.q, new r.z
  int* d_notspd = nullptr;           // [N + 1]
  int* d_ncols = nullptr;            // [N]
  int* d_mk = nullptr;               // [N] Krylov basis size at the last Rayleigh-Ritz
  int* d_nwk = nullptr;              // [N] wanted Ritz pairs
  // Waves: subdomains whose layer blocks, factors and solve buffers share one
  // pool of device memory, processed one wave after another by the local
  // stage (one wave holding every subdomain when everything fits).
  std::vector<WaveSched> waves;
  int cur = 0;                       // wave being processed
  std::vector<int> wave_of;          // [N] wave of each subdomain
  void* d_pool = nullptr;            // layer-block / solve-buffer pool
  size_t pool_bytes = 0;
  int mixed = 0;                     // precision == MSGFEM_MIXED
  int geneo = 0;                     // method == MSGFEM_METHOD_GENEO: the GenEO eigenproblem on Omega_j
  int factor_tc = 0;                 // FP32 factorisation on the tensor cores (msgfem_options.factor_kernel)
  void* d_tc_maps = nullptr;         // device tensor maps of every subdomain's FP32 arrays (4 per subdomain)
  void* d_solve_maps = nullptr;      // the same arrays in 64 x 64 unswizzled boxes (TMA solve stages)
  int* d_kerr = nullptr;             // set by a TMA solve stage that did not arrive in time
  int potrf_fp64 = 0;                // mixed: FP64 tile Cholesky after an FP32 one met a bad pivot
  int factor_persistent = 0;         // mixed: FP32 factorisation as one persistent launch
  int refine = 2;                    // FP64 refinement steps per FP32 solve
  std::vector<CoarsePair> pairs;
  CoarsePair* d_pairs = nullptr;
  double* d_pair_part = nullptr;
  int Nc = 0, NcPad = 0;
  std::vector<int> coff;
  int* d_coff = nullptr;
  int* d_m = nullptr;
  double* d_AH = nullptr;
  double* d_AHinv = nullptr;
  double* d_cscr = nullptr;   // scratch tiles of the coarse inverse's split rows
  double* d_cid = nullptr;    // identity strip [I I ... I] of the coarse inverse
  double* d_bH = nullptr;
  double* d_cH = nullptr;
  double* d_yH = nullptr;
  double* d_rH = nullptr;
  double* d_u = nullptr;
  double* d_ref = nullptr;
  double* d_energy = nullptr;
  double* d_l2 = nullptr;            // [1024][4] block sums of the L2 errors (msgfem_solution_errors)
  Schedule cfact;
  SolveSchedule csolve;
  int n_loc = 0, p = 0;              // n_loc: the largest nloc_j (columns of lam_host and of the bases)
  // profiling (CUDA events on the handle's stream)
  struct Span { int tag; cudaEvent_t a, b; };
  std::vector<Span> spans;
  std::vector<cudaEvent_t> ev_pool;
  msgfem_profile prof{};
  int stage = 0;   // 1 setup, 2 local spaces, 3 coarse assembled, 4 solved
  std::string err;
  // learned warm start
  std::vector<WarmStart> warm;       // [N] registered start blocks
  void* d_warm = nullptr;            // device descriptors of the start blocks
  std::vector<int*> d_b2rows;        // [N] ascending full-layout rows of B2
  // device current at msgfem_setup, and the address of the fixed scratch array of
  // msgfem_energy_error_noalloc on it
  int device = -1;
  double* noalloc_scratch = nullptr;
  // wave whose layer-block factors are resident in the pool (-1: none or stale)
  int factored_wave = -1;
  // a hexahedron-list mesh: structured id of every node / element of the list,
  // and on the device the same map, its inverse and a staging vector
  std::vector<int> node_of_user, elem_of_user;
  int* d_node_of_user = nullptr;
  int* d_user_of_node = nullptr;
  double* d_perm_tmp = nullptr;
  // two-level Schwarz PCG (msgfem_schwarz_solve): global vectors x, r, z, p, q
  // on all DoFs, partial sums of the dot products
  double* d_pcg_vec = nullptr;
  double* d_pcg_part = nullptr;
};

extern long long g_launch_count;   // kernel launches issued by this library

msgfem_status cuda_fail(msgfem* h, cudaError_t e, const char* what, const char* file, int line);
// device memory of the handle (msgfem_options.dev_alloc / dev_free, or cudaMalloc /
// cudaFree), recorded in h->allocs and released by msgfem_destroy
msgfem_status dev_alloc_bytes(msgfem* h, void** out, size_t bytes);
void dev_free_bytes(msgfem* h, void* p);

// host scheduling (setup.cpp)
msgfem_status build_problem(msgfem* h);
void build_factor_schedule(msgfem* h);
void build_wave_factor_schedule(msgfem* h, WaveSched& w);
void build_solve_schedules(msgfem* h);
void build_wave_solve_schedules(msgfem* h, WaveSched& w);
// the coarse schedules; with d_cscr and d_cid set, the block inverse's rows of
// more than COARSE_INV_SPLIT tiles are split into partial sums (setup.cpp)
void build_coarse_schedules(msgfem* h);
constexpr int COARSE_INV_SPLIT = 8;
// scratch tiles and identity-strip width (in tiles) the split needs for T tiles
void coarse_inverse_split_sizes(int T, int split, size_t* scratch_tiles, int* maxc);
// device storage of one subdomain's layer blocks, factors and solve buffers
// (bytes, and placement at base: pointers of sub[j] set), and the grouping of
// the subdomains into waves that fit the byte budget (h->waves, h->wave_of,
// h->pool_bytes = the largest wave)
size_t sub_block_bytes(msgfem* h, int j);
size_t place_sub_blocks(msgfem* h, int j, char* base);
msgfem_status plan_waves(msgfem* h, size_t budget);
// element types of the angle field h->h_angles (per ply, per element shape /
// frame / angle on curved meshes, or per element)
void element_types(const msgfem* h, bool& layered, std::vector<double>& types, std::vector<int>& etype,
                   std::vector<int>& trep);

// launchers
void set_dense_context(int* active, int* notspd, const SubDev* subs);
// FP32 factorisation kernel of the next schedule runs: the tensor-core tile
// kernel when tc_maps (device tensor maps of the subdomains' FP32 arrays) is
// given, else the SIMT one; potrf32: its 64 x 64 tile Cholesky in FP32 (else FP64)
void set_factor_kernel(const void* tc_maps, int potrf32);
// encode and upload h->d_tc_maps (k_dense.cu)
msgfem_status tc_maps_build(msgfem* h);
// the kernel choice of h for its next factorisation (tensor maps built on first use)
msgfem_status select_factor_kernel(msgfem* h);
void prepare_tile_kernels();
template <typename T>
void run_schedule(const ScheduleT<T>& s, cudaStream_t st, const StreamSet* gs = nullptr);
// solve steps; scatter_add adds the result into the destination multivector
enum { SOLVE_DEFAULT = 0, SOLVE_ASYNC_RING = 1, SOLVE_STREAM = 2, SOLVE_STREAM_CL2 = 3, SOLVE_TMA_RING = 4 };
// tensor maps and error flag of the TMA solve stages (k_dense.cu), set before solve runs
void set_solve_maps(const void* maps, int* err);
msgfem_status solve_maps_build(msgfem* h);
// MSGFEM_ECUDA (and the flag cleared) when a TMA solve stage reported a failure
msgfem_status check_stage_error(msgfem* h);
// allocate (once) and clear the device error flag of bounded waits (k_dense.cu)
msgfem_status kerr_ensure(msgfem* h);
// 1 when the FP32 factorisation's tile Cholesky runs in FP32 (k_dense.cu)
int tile_chol_fp32(const msgfem* h);
// the persistent FP32 factorisation of wave w on stream st (cooperative launch; k_dense.cu)
msgfem_status run_factor_persistent(msgfem* h, const WaveSched& w, cudaStream_t st);
// stream groups of the factorisation schedules: one per chain (persistent) or ngroup_factor
int factor_groups(const msgfem* h, const WaveSched& w);
template <typename T>
void run_solve_mv(const SolveScheduleT<T>& s, cudaStream_t st, int src, int dst, int gather_neg, int width = PST,
                  const StreamSet* gs = nullptr, int scatter_add = 0, int variant = SOLVE_DEFAULT);
void launch_element_stiffness(msgfem* h);
// Structured numbering of a hexahedron list (hexmesh.cpp): the (i, j, k) block
// dimensions and, for every node and element of the list, its structured id.
struct HexNumbering {
  int nx = 0, ny = 0, nz = 0;
  std::vector<int> node_of_user, elem_of_user;
};
bool recover_structure(int n_nodes, int n_elems, const int* hex8, HexNumbering& out, std::string& err);
// element boxes {x0, x1, y0, y1} of the parts of a structured element -> part map
bool parts_to_boxes(int NX, int NY, int NZ, const int* elem_part, std::vector<int>& boxes, std::string& err);
// per-node Dirichlet flags (structured order) equal to the clamped face i = 0
bool dirichlet_is_clamped_face(int NX, int NY, int NZ, const unsigned char* flags, std::string& err);

// general mesh input (k_numbering.cu): set-up through the structured path, and
// node-major vectors on all DoFs between the caller's numbering (host or
// device) and the structured one on the device; element angles into the
// structured order on the host
msgfem_status setup_general(const msgfem_mesh* mesh, const msgfem_plies* plies, const msgfem_partition* part,
                            int overlap, int oversampling, const msgfem_options* opt, msgfem_h* out);
msgfem_status vec_in(msgfem* h, const double* user, double* d_struct);
msgfem_status vec_out(msgfem* h, const double* d_struct, double* user);
msgfem_status angles_in(msgfem* h, const double* user, std::vector<double>& out);

// load vector on all DoFs (given nodal loads or the end-face traction), zero on
// the clamped face (setup.cpp)
std::vector<double> global_load(const msgfem* h);
// node coordinates of node (i, j, k): given, or those of the box (setup.cpp)
void node_xyz(const msgfem* h, int i, int j, int k, double X[3]);
void launch_stencil(msgfem* h);
void launch_layer_blocks(msgfem* h);
void launch_layer_blocks_f32(msgfem* h);
void launch_stencil_apply(msgfem* h, int src, int dst, int mode, double alpha);
void launch_gram(msgfem* h, int wx, int wy, int wg);
void launch_small_eig(msgfem* h, int p);
void launch_rotate(msgfem* h, int which, int wy, int ncols);
void launch_sub_rc(msgfem* h, int wout, int wr, int wc, int nr);
void launch_random_b2(msgfem* h, int which, int p, unsigned long long seed);
void launch_mask_rows(msgfem* h, int which, int keep);
void launch_zero_pins(msgfem* h, int which);
void launch_copy_col(msgfem* h, int wsrc, int scol, int wdst, int dcol, double sign);
void launch_copy_mv(msgfem* h, int wsrc, int wdst);
void launch_rigid_modes(msgfem* h);
void launch_chol_inv_small(msgfem* h, int wg, const int* d_ncols, int nfixed, int drop_last);
// relative residual per column c < p over the rows of the DoF classes in keep:
// ||A_c + sgn theta_c B_c|| / (||A_c|| + |theta_c| ||B_c||) into resid
void launch_colnorms(msgfem* h, int wa, int wb, int p, int keep = 1 << 2, double sgn = 1.0);
void launch_scale_rows_mu(msgfem* h, int which);
void launch_theta_axpy(msgfem* h, int wx, int wy, int wd, int p);
void launch_x_minus_y(msgfem* h, int wx, int wy, int wd, int stride);
void launch_sub_load_kb(msgfem* h, int which);
// preconditioned CG of the mixed-precision K solves (KB-wide blocks): masked
// column dots into slot `slot` of d_pcg, and the vector updates
void launch_coldot_kb(msgfem* h, int wx, int wy, int keep, int slot);
enum { PCG_STEP = 0, PCG_DIR = 1, PCG_DIR0 = 2 };
void launch_pcg_update(msgfem* h, int mode, int wx, int wr, int wz, int wp, int wq);
// adaptive refinement: clear the active flag of subdomains whose residual
// block wr (rows of the DoF classes in the bit mask keep) is converged or
// stagnant (step -1 records the reference norm)
void launch_refine_check(msgfem* h, int wr, int wref, int keep, int step);
constexpr int KEEP_K = (1 << 1) | (1 << 2);   // rows of K: B1 and B2
constexpr int KEEP_A11 = 1 << 1;               // rows of A11: B1
#ifndef MSGFEM_REFINE_TOL
#define MSGFEM_REFINE_TOL 1e-13
#endif
constexpr double REFINE_TOL = MSGFEM_REFINE_TOL;   // relative residual at which refinement stops
// relative residual at which the conjugate-gradient K solves of the mixed path stop
// (the eigensolver's own tolerance is 1e-7 in the energy norm)
constexpr double PCG_TOL = 1e-11;
void launch_refine_check_tol(msgfem* h, int wr, int wref, int keep, int step, double tol);
void launch_coarse_blocks(msgfem* h);
void launch_coarse_rhs(msgfem* h);
void launch_prolong(msgfem* h);
int energy_blocks(msgfem* h);
void launch_energy(msgfem* h, const double* d_ref, const double* d_u, double* d_out);
void launch_basis_out(msgfem* h, int j, double* d_out, int ncols);
// one vector of subdomain j between the internal layout and that of
// msgfem_get_basis (to_output 1: internal -> output)
void launch_vec_layout(msgfem* h, int j, const double* src, int sstride, double* dst, int dstride, int to_output);

// two-level Schwarz PCG (k_schwarz.cu): factors of a one-wave handle made
// resident, and the A11 solve of the KB-wide working blocks (TB -> WB)
msgfem_status schwarz_factors(msgfem* h);
void schwarz_local_solve(msgfem* h);

// msgfem_energy_error_noalloc (k_noalloc.cu): resolve its fixed array on the
// current device (called by msgfem_setup)
msgfem_status noalloc_prepare(msgfem* h);

// learned warm start (k_warm.cu)
msgfem_status warm_rows(msgfem* h);
bool warm_upload(msgfem* h);
msgfem_status warm_check(msgfem* h, std::vector<int>& bad);
void launch_load_start(msgfem* h, int which);

// error helpers shared by the translation units that return msgfem_status
#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return cuda_fail(h, e_, #x, __FILE__, __LINE__); } while (0)
#define CK_LAUNCH() CK(cudaGetLastError())
#define TRY(x) do { msgfem_status st_ = (x); if (st_ != MSGFEM_OK) return st_; } while (0)

// source selectors for k_copy_col
enum { SRC_BLOAD = -1, SRC_PSI = -2 };

#ifdef __CUDACC__
__device__ __forceinline__ double* mv_ptr(const SubDev& s, int which) {
  switch (which) {
    case MV_PHI: return s.Phi;
    case MV_Z: return s.Z;
    case MV_KPHI: return s.KPhi;
    case MV_W: return s.W;
    case MV_T1: return s.T1;
    case MV_R: return s.R;
    case MV_BR: return s.BR;
    case MV_EV: return s.EV;
    case MV_CB: return s.CB;
    case MV_CW: return s.CW;
    case MV_QB: return s.QB;
    case MV_NQ: return s.NQ;
    case MV_ZB: return s.Zb;
    case MV_WB: return s.Wb;
    case MV_P1: return s.P1;
    case MV_P2: return s.P2;
    case MV_P3: return s.P3;
    default: return s.Tb;
  }
}
__device__ __forceinline__ int mv_stride(int which) {
  return (which == MV_QB || which == MV_NQ) ? MQ : (which >= MV_ZB ? KB : PST);
}
__device__ __forceinline__ double* gm_ptr(const SubDev& s, int which) {
  switch (which) {
    case GM_G1: return s.G1;
    case GM_G2: return s.G2;
    case GM_G3: return s.G3;
    default: return s.Y;
  }
}
#endif
