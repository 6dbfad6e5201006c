// Internal data structures shared by the host engine and the sm_103a kernels.
//
// Vector layout ("padded"): a level with n interior nodes per axis stores P^d
// elements, P = n + 1, with interior node (x, y, z) (0-based, < n) at
// (z * P + y) * P + x.  Positions with a coordinate equal to n are ghosts and hold
// zero; every kernel that writes a vector writes zero there.  P is a power of two for
// n = 2^L - 1, so rows are aligned.  Kernels bounds-check every neighbour load, so
// nothing outside [0, P^d) is ever touched.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <string>

#ifdef __CUDACC__
#define HELM_HD __host__ __device__
#else
#define HELM_HD
#endif

namespace helm {

constexpr int SMAX = 4;            // max GMRES(s) steps per smoothing sweep
constexpr int NPART = 2 * SMAX + 4;  // doubles per partial-sum slot of a sweep pass

// Real and complex scalar types of a preconditioner precision.
template <typename C> struct RealOf;
template <> struct RealOf<float2> { typedef float T; };
template <> struct RealOf<double2> { typedef double T; };
template <typename R> struct CplxOf;
template <> struct CplxOf<float> { typedef float2 T; };
template <> struct CplxOf<double> { typedef double2 T; };

// Per (problem, level) state of the current GMRES(s) sweep, device memory, in the
// working precision R of the V-cycle (FP32 for complex64: nothing in that V-cycle
// touches the slow FP64 pipe).  Raw vectors R_0 = r0 (initial residual of the
// sweep), R_j = p_j = M v_j.  Every Arnoldi vector is kept as coefficients over the
// raw vectors:  v_j = sum_{k<j} Cf[j][k] R_k   (j = 1..s).
template <typename R>
struct SweepScalarsT {
  typedef typename CplxOf<R>::T CR;
  R beta2;                        // ||R_0||^2
  int m;                          // Krylov steps of this sweep (0: nothing to do)
  int s;                          // requested steps
  CR Cf[SMAX + 1][SMAX + 1];      // Arnoldi vectors over raw vectors
  CR Hh[SMAX + 1][SMAX];          // Hessenberg matrix of the sweep
  CR xcoef[SMAX + 1];             // x_new = x_old + sum_k xcoef[k] R_k
  CR rcoef[SMAX + 1];             // r_new = sum_k rcoef[k] R_k
  int status;                     // nonzero: NaN/Inf seen
  int pad0;
  // everything above is the sweep algebra's state (staged through shared memory);
  // the reduction counter below is never part of that copy
  unsigned int counter;           // last-block-done counter
  int pad1;
};

// One level of one problem, as seen by the kernels (device memory).
template <typename C>
struct LevelDev {
  int n, P;               // interior nodes per axis, pitch n+1
  int nc, Pc;             // next coarser level (0 on the coarsest)
  int ntiles;             // tiles of this level per problem (for reductions)
  int s;                  // GMRES steps per sweep
  C* b;                   // right-hand side of this level
  C* xa;                  // iterate after pre-smoothing
  C* xb;                  // iterate after coarse correction and post-smoothing (output)
  C* r0;                  // initial residual of a post-smoothing sweep
  C* p[SMAX];             // p_j = M v_j
  C* bc;                  // coarser level's b (restriction target)
  const C* xcb;           // coarser level's output (prolongation source)
  const C* ca;            // 1D coefficients of u_{i-1}  (length n)
  const C* cd;            // 1D coefficients of u_i      (= ca + n)
  const C* cc;            // 1D coefficients of u_{i+1}  (= ca + 2n)
  const float* phi;       // phi field in padded layout, or nullptr
  double phic;            // constant phi when phi == nullptr
  typename RealOf<C>::T phir;  // phic rounded to the level's precision (no conversion per point)
  SweepScalarsT<typename RealOf<C>::T>* sc;   // this level's sweep state
  SweepScalarsT<typename RealOf<C>::T>* scc;  // coarser level's sweep state
  double* part;           // partial sums: ntiles * NPART slots (R or double)
  const CUtensorMap* tm;  // 2D complex64 levels: TMA maps of b, r0, p_1..p_SMAX (else nullptr)
};

// TMA maps per level: b, r0, p_1..p_SMAX (in this order).
constexpr int TM_B = 0, TM_R0 = 1, TM_P0 = 2, TM_XB = 2 + SMAX, TM_COUNT = 3 + SMAX;

// Dense LU factors of the coarsest operator (FP64), row-major, with pivots.
constexpr int MAX_COARSE_LEVELS_HOST = 8;  // levels the staged coarse kernels hold

struct CoarseLU {
  int m;                  // unknowns (n^d)
  int nlev;               // levels of the problem's coarse sub-cycle
  const double2* lu;      // m*m
  const int* piv;         // m
};

// Outer FGMRES state of one problem (FP64, device memory).
struct OuterState {
  int j;                  // index of the Arnoldi vector being preconditioned
  int m;                  // restart length (columns of Hbar)
  int iters;              // total preconditioner applications
  int maxit;
  int done;               // 0 running, 1 converged, 2 maxit, 3 numeric, 4 breakdown
  int cycle_end;          // 1: the current cycle must end (solve and recompute)
  int restarts;
  int status;
  double tol;
  double bnorm;           // ||b||
  double beta;            // ||r0|| of the current cycle
  double rel_est;         // |g_{j+1}| / ||b||
  double rel_true;        // last true relative residual
  double hnext;           // h_{j+1,j} of the last column
  double wnorm2;          // ||w||^2 of the last column
  unsigned int counter;   // last-block counter
  int need_residual;      // 1: the true residual must be recomputed (start or cycle end)
  int fresh;              // 1: a new cycle starts, v_0 must be formed
  int df;                 // 1: the Krylov basis and H z_j are held and reduced in double-float
};

// Per-problem pointers of the outer solve (device memory).
template <typename C>
struct OuterDev {
  int n, P, ntiles;
  const double2* ca; const double2* cd; const double2* cc;  // H coefficients
  const float4* cdf;      // the same as double-floats: a, d, c blocks of n
  const float* phi; double phic;
  double2* bpad;          // b in padded layout
  double2* xpad;          // x in padded layout
  double2* w;             // scratch: H z_j, then residual
  double2* V;             // (m+1) Arnoldi vectors, padded, stride vs
  C* Z;                   // m preconditioned vectors, padded, stride vs
  C* b0;                  // V-cycle input of level 0 (precision C)
  const C* zout;          // V-cycle output of level 0 (precision C)
  int s;                  // GMRES steps per smoothing sweep
  size_t vs;              // elements per vector (P^d)
  double2* Hm;            // (m+1) x m Hessenberg, column-major
  double2* g;             // m+1
  double* cs; double2* sn;// Givens rotations
  double2* y;             // m
  double2* hcol;          // m+1 reduced dots of the current column
  double* vscale;         // m+1: v_i = vscale[i] * V[i] (V stored unnormalised)
  double* part;           // partial sums
  unsigned* gcnt;         // the multi-dot's group counters (zero between calls)
  OuterState* st;
  SweepScalarsT<typename RealOf<C>::T>* sc0;  // level-0 sweep state (set by the kernel that writes b0)
};

// Tile configuration: rows (2D) or planes (3D) marched per warp / CTA (even).
struct TileCfg {
  int rows;
  int P = 0;   // pitch of the level (n + 1)
};

constexpr int WARPS2 = 8;     // 2D: warps per CTA (each marches its own rows)
constexpr int WY3 = 8;        // 3D: owned y rows per CTA (plus 2 halo warps)

HELM_HD inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// V-cycle tile kernels: 2D tiles of 64 x 16 points; 3D blocks of 32 x 8 columns
// marching zchunk(P) planes.
HELM_HD inline int zchunk(int P) { return P >= 128 ? 32 : (P >= 64 ? 4 : 2); }
HELM_HD inline int vtiles(int dim, int P) {
  return dim == 2 ? ceil_div(P, 64) * ceil_div(P, 16) : ceil_div(P, 32) * ceil_div(P, 8) * ceil_div(P, zchunk(P));
}

// Marching FP64 stencil of the outer solve: 2D warps march cfg.rows rows, 3D CTAs
// march cfg.rows planes.
inline int tiles_per_problem(int dim, int P, TileCfg cfg) {
  if (dim == 2) return ceil_div(P, 32) * ceil_div(P, WARPS2 * cfg.rows);
  return ceil_div(P, 32) * ceil_div(P, WY3) * ceil_div(P, cfg.rows);
}

// ---------------------------------------------------------------- persistent V-cycle segments
// Passes of the small grid-wide levels walked by one cooperative launch (tiles.cuh
// k_vcycle_seq): each pass's virtual blocks are the blocks of its ordinary launch.
enum PassKind { PK_ARNOLDI = 0, PK_RESTRICT = 1, PK_PROLONG = 2, PK_UPDATE = 3, PK_PROLONG_FLAT = 4 };
struct PassDesc {
  const void* levs;  // the depth's LevelDev array (device)
  int kind, J;
  int ntiles;        // tiles (marching passes) or flat blocks per problem
  int geo;           // 2D tiles per CTA, 3D planes per march
  int f0, f1, f2, f3;  // kind-specific flags (see run_pass)
  int nvblk;         // virtual blocks of the pass over all problems
};
constexpr int SEQ_MAX = 56;
struct PassSeq {
  int npass;
  PassDesc p[SEQ_MAX];
};
static_assert(sizeof(PassSeq) <= 4000, "the pass list travels as a kernel argument");

// Grid barrier of the persistent launch: arrival count and generation, cleared before
// every launch.
struct GridBar {
  unsigned count, gen;
};
// ---------------------------------------------------------------- launchers
enum UpdateMode { UPD_RESTRICT = 0, UPD_RESIDUAL = 1, UPD_XONLY = 2 };

// V-cycle passes (vcycle_c64.cu / vcycle_c128.cu), C = float2 or double2.
template <typename C>
void launch_arnoldi(int dim, int J, const LevelDev<C>* levs, int nprob, int ntiles, TileCfg cfg, bool r0_is_b,
                    bool store_p, bool tma, cudaStream_t st);
template <typename C>
void launch_restrict(int dim, const LevelDev<C>* levs, int nprob, int ntiles, TileCfg cfg, bool r0_is_b,
                     bool x_from_zero, bool nosmooth, cudaStream_t st, bool tma = false, int nraw = SMAX + 1);
template <typename C>
void launch_update_flat(int dim, UpdateMode mode, const LevelDev<C>* levs, int nprob, int ntiles, bool r0_is_b,
                        int xsel, bool x_from_zero, cudaStream_t st);
template <typename C>
void launch_prolong(int dim, bool with_residual, const LevelDev<C>* levs, int nprob, int ntiles, TileCfg cfg,
                    bool tma, cudaStream_t st);
// Recorders of the same passes into a pass list, and the cooperative launch of a list.
template <typename C>
void record_arnoldi(PassSeq& q, int dim, int J, const LevelDev<C>* levs, int nprob, int ntiles, TileCfg cfg,
                    bool r0_is_b, bool store_p);
template <typename C>
void record_restrict(PassSeq& q, int dim, const LevelDev<C>* levs, int nprob, int ntiles, TileCfg cfg, bool r0_is_b,
                     bool x_from_zero, bool nosmooth);
template <typename C>
void record_update(PassSeq& q, int dim, UpdateMode mode, const LevelDev<C>* levs, int nprob, int ntiles, bool r0_is_b,
                   int xsel, bool x_from_zero);
template <typename C>
void record_prolong(PassSeq& q, int dim, bool with_residual, const LevelDev<C>* levs, int nprob, int ntiles,
                    TileCfg cfg);
template <typename C>
int launch_seq(int dim, const PassSeq& q, GridBar* gb, unsigned long long limit_ns, cudaStream_t st);
template <typename C>
void launch_coarse(int dim, const LevelDev<C>* levs, int nlev, int lev_stride, const CoarseLU* lus, int nprob,
                   int nu1, int nu2, cudaStream_t st);
// coarse sub-cycle staged in shared memory (smem_bytes: all levels' vectors)
template <typename C>
void launch_coarse_cluster(int dim, const LevelDev<C>* levs, int lev_stride, const CoarseLU* lus, int nprob,
                           int nu1, int nu2, cudaStream_t st);
template <typename C>
void launch_coarse_smem(int dim, const LevelDev<C>* levs, int nlev, int lev_stride, const CoarseLU* lus, int nprob,
                        int nu1, int nu2, size_t smem_bytes, cudaStream_t st);
// level-0 input from a natural-layout vector of precision in_prec (HELM_C64/HELM_C128)
template <typename C>
void launch_load_input(int dim, const LevelDev<C>* levs, int ntiles, const void* src, int in_prec, cudaStream_t st);
template <typename C>
void launch_store_output(int dim, int n, const LevelDev<C>* levs, void* dst, int out_prec, cudaStream_t st);

// Outer FP64 kernels (outer.cu).
template <typename C>
void outer_residual(int dim, const OuterDev<C>* od, int nprob, int ntiles, TileCfg cfg, cudaStream_t st);
template <typename C>
void outer_apply_h(int dim, const OuterDev<C>* od, int nprob, int ntiles, TileCfg cfg, cudaStream_t st);
// TMA maps of a 2D complex64 level (tma.cpp): a 136 x 18 float box (64 x 16 complex
// points plus halo) over a P x P complex field.  False when the driver has no
// tensor-map encoder or the layout does not meet its rules.
bool encode_level_tmaps(int P, const void* const* vectors, int count, CUtensorMap* out);
// TMA maps of a 3D complex64 level (tma.cpp): 72 x box_rows x 1 float boxes (a 32-point
// wide column tile plus halo, one plane) over a P^3 complex field; P a multiple of 32.
bool encode_level_tmaps3(int P, int box_rows, const void* const* vectors, int count, CUtensorMap* out);
// ---------------------------------------------------------------- tuned launch choices
// (tune.cpp) keyed by pass, dimension, level pitch P, precision (bytes per complex
// value) and Arnoldi step J (0 for the other passes); TUNE_NV integers per choice:
//   arnoldi (step J) and prolong (J = 0), 3D, complex64: {TMA-fed pass on, plane slots
//                            in flight, z pieces per column (0: one equal share per
//                            resident CTA), points per thread in y (2 or 4; 0: 2)}
//   arnoldi / restrict / prolong, 2D: {tiles per CTA}
//   persist, 2D/3D: {grid-wide level run inside the persistent segments (1) or by its
//                    own launches (0)}
enum TunePass { TP_ARNOLDI = 0, TP_RESTRICT = 1, TP_PROLONG = 2, TP_PERSIST = 3, TP_ZPLANES = 4 };
constexpr int TUNE_NV = 4;
struct TuneChoice {
  int v[TUNE_NV];
};
constexpr int TM3_STAGES_MAX = 8;     // plane slots of the 3D TMA-fed pass
// Read a table (path NULL: $HELM_TUNING, else tuning.json beside the library); replaces
// the current one.  Entries tuned on another kind of device are dropped.
int tune_load(const char* path, std::string* err);
void tune_load_default();             // once per process (helm_setup)
bool tune_get(int pass, int dim, int P, int prec_bytes, int J, TuneChoice* out);
void tune_set(int pass, int dim, int P, int prec_bytes, int J, const TuneChoice* c);  // NULL: remove
int tune_entries();
// Write the current table with the kept run records and `run_record` appended.
int tune_write(const char* path, const std::string& run_record, std::string* err);
// 2D tiles per CTA of a pass: the tuned value, else the heuristic's.
int tuned_tpc(int pass, int P, int prec_bytes, int J, int heuristic);
// Planes each CTA of the plain 3D passes (Arnoldi, restriction, prolongation) marches on
// a level of pitch P: the table's choice (2, 4, 8 or 16), else zchunk(P).
int tuned_zchunk(int P, int prec_bytes);
// Whether a grid-wide level of pitch P runs inside the persistent segments: only where
// the tuning table switches it on, for 2D levels up to 511^2 and 3D levels up to 63^3.
bool persist_level(int dim, int P, int prec_bytes);
// Spin limit of the persistent segments' grid barrier (helm_set_barrier_timeout; 1 s).
unsigned long long barrier_limit_ns();
void set_barrier_limit_ns(unsigned long long ns);

// The 3D TMA-fed Arnoldi pass of step J on a level of pitch P: whether it runs (else
// the plain pass), plane slots in flight, how the level is shared among CTAs (pieces
// > 0: every column in that many equal z pieces, one per CTA; 0: one equal share of
// the (column, plane) sequence per resident CTA), and points per thread in y (2, 4).
struct Tma3Params {
  bool enabled;
  int stages, pieces, qy;
};
Tma3Params tma3_params(int pass, int J, int P);  // pass TP_ARNOLDI (step J) or TP_PROLONG (J = 0)
constexpr int TMA3_MAX_UNITS = 2048;  // shares per problem (partial-sum slots of a 3D level)
constexpr int TMA3_MIN_P = 128;       // the 3D TMA-fed passes run on levels of 127^3 and larger
constexpr int TMA3_MAX_P = 1024;      // (32-bit point indices)
// Kernels of the coarse correction of a level: 2 where a 3D complex64 level splits it
// into the row-wise prolongation and the TMA-fed residual pass, else 1.
inline int prolong_kernels(int dim, bool with_residual, int prec_bytes, bool tma, int P) {
  return dim == 3 && with_residual && prec_bytes == 8 && tma && P >= TMA3_MIN_P && P <= TMA3_MAX_P &&
                 tma3_params(TP_PROLONG, 0, P).enabled
             ? 2
             : 1;
}
// Sticky device error flag of the V-cycle kernels (a wait ran out): read and clear.
int vcycle_take_error();
int vcycle_take_error_c128();
int outer_chunks(size_t vs);
size_t outer_part_doubles(int chunks, int m);
int outer_dot_counters(int chunks);
void basis_store(const double2* src, double2* dst, size_t n, int df, cudaStream_t st);
template <typename C>
void outer_dots(const OuterDev<C>* od, int nprob, int chunks, int m, size_t vs, cudaStream_t st);
template <typename C>
void outer_vnew(const OuterDev<C>* od, int nprob, int chunks, int m, bool start, cudaStream_t st);
template <typename C>
void outer_backsolve(const OuterDev<C>* od, int nprob, cudaStream_t st);
template <typename C>
void outer_solution(const OuterDev<C>* od, int nprob, int chunks, int m, cudaStream_t st);
// dst[p] = *src[p] for p < count (device pointers).
void gather_states(OuterState* const* src, OuterState* dst, int count, cudaStream_t st);

// Layout conversions and the stand-alone operator (convert.cu).
void convert_dense_to_padded_c128(int dim, int n, const double2* src, double2* dst, cudaStream_t st);
void convert_padded_to_dense_c128(int dim, int n, const double2* src, double2* dst, cudaStream_t st);
void scatter_phi(int dim, int n_level, int stride, int n_fine, const float* phi_dense_fine, float* phi_pad_level,
                 cudaStream_t st);
// w = A v on the finest level, A given by 1D coefficients (prec: HELM_C64/HELM_C128),
// natural layout in and out.
void apply_operator_dense(int dim, int n, const double2* ca, const double2* cd, const double2* cc,
                          const float* phi_pad, double phic, const void* v, void* w, int prec, cudaStream_t st);

}  // namespace helm
