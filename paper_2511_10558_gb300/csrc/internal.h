// Internal declarations shared by the host network compiler, the kernels and
// the C ABI glue. Not part of the public interface (include/carbox.h).
#pragma once

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "carbox.h"

namespace cbx {

constexpr int kMaxOrder = 5;           // BDF orders 1..5
constexpr int kDiffRows = kMaxOrder + 3;  // difference array rows D[0..q+2]
constexpr int kSegLen = 16;            // entries per right-hand-side gather segment
constexpr int kNumTypes = 4;           // CBX_TWO_BODY .. CBX_CR_PHOTO

// Device view of a compiled network: all species indices are internal
// (fill-reducing order); perm maps internal -> user index.
struct DevNet {
  int S, R, nnzJ, nseg;
  int kdense;            // pivots k >= kdense are factored over the full index ranges
  int sparse_panels;     // leading 32-wide panels whose trailing update the FP64 blocked LU takes from the lists
  const int* rtype;      // [R]
  const double* alpha;   // [R]
  const double* beta;    // [R]
  const double* gamma;   // [R]
  const int* ra;         // [R] first reactant
  const int* rb;         // [R] second reactant or -1
  const int* seg_ptr;    // [nseg+1] entry range of each gather segment
  const int* spec_seg;   // [S+1] segment range of each species
  const int* rhs_ent;    // (reaction << 1) | negative, |nu| copies per term
  const int* jrow;       // [nnzJ] row of each Jacobian slot (slots sorted by row, col)
  const int* jcol;       // [nnzJ] column
  const int* jrow_ptr;   // [S+1] CSR row pointer over the slots
  int njg;               // Jacobian gather groups of 32 slots
  const int* jg_ptr;     // [njg+1] term range of each group (a multiple of 32)
  const int* jg_slot;    // [32 njg] slot of each (group, lane), -1 past nnzJ
  const int* jg_len;     // [32 njg] terms of that slot
  const int* jg_term;    // term e of (group g, lane l) at jg_ptr[g] + 32 e + l:
                         // ((2 reaction + reactant slot) << 1) | negative
  const int* piv_lptr;   // [S+1] range of rows i > k with L(i,k) structurally non-zero
  const int* piv_l;
  const int* piv_uptr;   // [S+1] range of columns j > k with U(k,j) structurally non-zero
  const int* piv_u;
  const int* perm;       // [S] internal -> user species index
  const int* rprod;      // [4R] products of each reaction (internal), -1 absent
  // Reactions grouped by rate type, so that each type's rate coefficients are
  // evaluated in a loop of its own: group t is positions tptr[t]..tptr[t+1]-1;
  // position e holds reaction rj[e] with its beta and gamma in gbeta[e], ggamma[e].
  int tptr[kNumTypes + 1];
  const int* rj;         // [R]
  const double* gbeta;   // [R]
  const double* ggamma;  // [R]
  double albedo_factor;  // 1 / (1 - omega) of the cosmic-ray-induced photo form
};

// Forward trajectory recorded for the adjoint: per cell the program of
// difference-array operations and the result y of every accepted step.
struct TapeDev {
  int cap_ops = 0, cap_steps = 0;
  int* nops = nullptr;     // [C] ops recorded
  int* ops_kq = nullptr;   // [C][cap_ops] (kind << 8) | q; kind 0 init, 1 rescale, 2 step
  double* ops_v = nullptr; // [C][cap_ops] h0 (init), rho (rescale), h (step)
  double* ys = nullptr;    // [C][cap_steps][S] step results, internal species order
  double* ts = nullptr;    // [C][cap_steps] t_new of each recorded step
};

enum { kOpInit = 0, kOpRescale = 1, kOpStep = 2 };

// Host-side compiled network.
struct HostNet {
  int S = 0, R = 0, nnzJ = 0, nnzLU = 0, nseg = 0, kdense = 0;
  int head_ints = 0;  // 2 (kdense + 1) + entries of the sparse pivots' lists
  int sparse_panels = 0;  // see DevNet
  double lu_flops = 0;
  std::vector<int> perm, iperm, rprod;
  std::vector<int> rtype, ra, rb;
  std::vector<double> alpha, beta, gamma;
  std::vector<int> seg_ptr, spec_seg, rhs_ent;
  std::vector<int> jrow, jcol, jrow_ptr;
  int njg = 0;
  std::vector<int> jg_ptr, jg_slot, jg_len, jg_term;
  std::vector<int> piv_lptr, piv_l, piv_uptr, piv_u;
  int tptr[kNumTypes + 1] = {};
  std::vector<int> rj;
  std::vector<double> gbeta, ggamma;
  double albedo = 0.0;  // omega
};

// Returns "" on success, else an error message.
std::string compile_network(const cbx_species* sp, int S, const cbx_reaction* rx, int R, HostNet* out);

// Minimum-degree ordering of a symmetric pattern (adjacency as dense bool, S x S).
std::vector<int> minimum_degree_order(const std::vector<uint8_t>& sym, int S);

struct SolveArgs {
  DevNet net;
  const double* alpha;  // [R] device: the alpha values of this solve (the network's, or a per-call set)
  const cbx_cell_params* phi;
  const double* x0;
  int C;
  double t0, t_end;
  double rtol, atol, newton_tol, refine_tol;
  int max_steps, max_refine;
  double gam[kMaxOrder + 2];  // gamma_q = sum_{j=1..q} 1/j
  double* x_out;
  int* status;
  cbx_cell_stats* stats;
  TapeDev tape;    // recording target (tape.nops == nullptr: no recording)
  double* ws;      // per-CTA workspace, ws_stride doubles per CTA
  long long ws_stride;
  int* counter;    // next-cell counter, zero before the launch
  int piv_ints;    // pivot-list ints staged in shared memory (set by launch_solver)
  const double* track;  // [C][K][6] (t, n_H, T, A_V, G0, zeta) knots, or null: phi is constant
  int K;
  const double* t_end_cell;  // [C] per-cell end times (device), or null: t_end for every cell
  // ESDIRK tableau (CBX_METHOD_ESDIRK): A [5][5] lower triangular, c [5], gamma = A[i][i], i >= 1
  double rk_a[5][5];
  double rk_c[5];
};

// The ESDIRK 4(3) of Kvaerno's family (explicit first stage, stage order 2,
// embedded and final solutions as stages 4 and 5, L-stable), derived on the
// host from those conditions; computed once.
struct EsdirkTableau {
  double a[5][5];
  double c[5];
  double gamma;
};
const EsdirkTableau& esdirk_tableau();

struct GradArgs {
  DevNet net;
  const double* alpha;  // [R] device: the alpha values of the recorded solve
  TapeDev tape;
  const cbx_cell_params* phi;  // [C] as recorded (constant environment), or null with a track
  const double* track;         // [C][K][6] the recorded solve's environment tracks, or null
  int K;
  double t0;                   // start time of the recorded solve
  const int* status;           // [C] forward status
  const double* x0;            // [S][C] as recorded (user order)
  const double* cot;           // [S][C] dL/dx(t_end) (user order)
  int C;
  double gam[kMaxOrder + 2];
  double* gcell;               // [C][R] per-cell dL/d ln alpha
  double* g_lognH;             // [C] or null
  double* g_T;                 // [C] or null
  double* ws;                  // per-CTA workspace, ws_stride doubles per CTA
  long long ws_stride;
  int* counter;
};

// Adjoint launch: workspace doubles per CTA, CTAs per SM, launch.
long long grad_workspace_doubles(int S, int R, int nnzJ);
int grad_occupancy(int S, int R, int nseg);
int launch_grad(const GradArgs& a, int grid, void* stream);
int launch_reduce_cells(const double* gcell, int C, int R, double* out, void* stream);
// Per-cell dL/d ln zeta, dL/d ln G0, dL/dA_V from gcell (outputs may be null).
int launch_env_grad(const double* gcell, int C, const DevNet& n, double* g_lnzeta, double* g_lnG0, double* g_AV,
                    void* stream);

// Launch plan of the solver kernel for one network and precision: matrix in
// shared memory (gm = false) or in the CTA's global workspace (gm = true).
struct SolverPlan {
  bool mixed = false, gm = false;
  size_t smem = 0;          // dynamic shared memory per CTA
  long long ws_stride = 0;  // per-CTA global workspace, in doubles
  int occupancy = 0;        // CTAs per SM (0: cannot launch)
  int piv_ints = 0;         // staged pivot-list ints in shared memory (0: none)
};
size_t smem_bytes(int S, int R, int nseg, bool mixed, bool gm, int piv_ints = 0);
long long workspace_doubles(int S, int R, int nnzJ, bool mixed, bool gm);
SolverPlan plan_solver(int S, int R, int nseg, int nnzJ, bool mixed, int head_ints);
// Launch the solver; returns a cudaError_t value.
int launch_solver(const SolveArgs& a, const SolverPlan& p, int grid, void* stream);
// One translation unit per kernel instantiation (precision x matrix placement).
int launch_solve_fp64(const SolveArgs& a, size_t smem, int grid, void* stream);
int launch_solve_fp64_gm(const SolveArgs& a, size_t smem, int grid, void* stream);
int launch_solve_mixed(const SolveArgs& a, size_t smem, int grid, void* stream);
int launch_solve_mixed_gm(const SolveArgs& a, size_t smem, int grid, void* stream);
int occupancy_solve_fp64(size_t smem);
int occupancy_solve_fp64_gm(size_t smem);
int occupancy_solve_mixed(size_t smem);
int occupancy_solve_mixed_gm(size_t smem);
int launch_solve_fp64_rk(const SolveArgs& a, size_t smem, int grid, void* stream);
int launch_solve_mixed_rk(const SolveArgs& a, size_t smem, int grid, void* stream);
int launch_solve_fp64_gm_rk(const SolveArgs& a, size_t smem, int grid, void* stream);
int launch_solve_mixed_gm_rk(const SolveArgs& a, size_t smem, int grid, void* stream);
// Launch the ESDIRK solver; returns a cudaError_t value.
int launch_solver_rk(const SolveArgs& a, const SolverPlan& p, int grid, void* stream);
int device_sm_count();
// cbx_solve on device buffers with at most max_grid CTAs (0: no cap) and,
// optionally, per-cell end times t_end_cell [C] (device; t_end must then be
// their maximum).
int solve_device(cbx_network* net, const cbx_cell_params* phi, const double* x0, int C, double t0, double t_end,
                 const cbx_options* opt, void* stream, double* x_out, int* cell_status, int max_grid,
                 const double* t_end_cell = nullptr);
// Set the calling thread's cbx_last_error() message; returns code.
int record_error(int code, const std::string& msg);
size_t device_smem_optin();

}  // namespace cbx

// Library-side network object behind the opaque cbx_network handle.
struct cbx_network {
  cbx::HostNet host;
  cbx::DevNet dev;
  void* dbuf = nullptr;  // one device allocation holding every table
  int device = 0;
  std::mutex mu;
};
