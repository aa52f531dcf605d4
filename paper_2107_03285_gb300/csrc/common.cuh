// Internal declarations of libsgn: the context, device views of the symbolic
// data, and the kernel launchers shared by the translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "../../include/sgn.h"
#include "symbolic.h"

namespace sgn {

// outer block of the factorization: Bunch-Kaufman panels (width = the
// setup's panel) are grouped into blocks of this many columns; the trailing
// Schur update runs once per block with an inner dimension of this size
constexpr int FACTOR_BLOCK = 256;

// device status word bits (sticky until read by a synchronising call)
enum : int {
  DEV_INVERTED = 1,
  DEV_NONFINITE = 2,
  DEV_TIMEOUT = 4,   // a bounded device-side wait expired
};

// device views of the static symbolic data
struct DevSym {
  int dim = 0, n_nodes = 0, n_elem = 0, n_free = 0, n_sn = 0, panel = 32;
  const int32_t *elem_node = nullptr, *elem_rank = nullptr;
  const double *elem_B = nullptr, *elem_vol = nullptr;
  const double *X = nullptr;               // rest positions [n_nodes][dim]
  const int32_t *node_rank = nullptr, *rank_node = nullptr;
  const int32_t *bsr_ptr = nullptr, *bsr_col = nullptr, *bsr_orig_pos = nullptr;
  const int32_t *up_slot = nullptr, *up_slot_t = nullptr, *up_ptr = nullptr, *up_contrib = nullptr;
  const int32_t *inc_ptr = nullptr, *inc = nullptr;
  const int32_t *sn_first = nullptr, *sn_nown = nullptr, *sn_nstruct = nullptr;
  const int32_t *sn_child_off = nullptr, *sn_nchild = nullptr;
  const int64_t *sn_struct_off = nullptr;
  const int32_t *struct_ranks = nullptr, *relpos = nullptr, *children = nullptr;
  const int64_t *cmap_off = nullptr;
  const int32_t *cmap = nullptr;
  const int32_t *lvl_fronts = nullptr;     // concatenated per-level lists (sorted by nown desc)
  const int32_t *item_sn = nullptr, *item_P = nullptr;  // per-level (front, node column) items
};

// one band or block of a front in a level's substitution schedule: q indexes
// the level-ordered front list, key orders the work inside the front
// (backward: key < 0 is a part of an ancestor-row product, see bwd_parts)
struct SolveItem {
  int32_t q, key;
};

// Backward substitution of an FP32 front with many ancestor (struct) rows:
// the product of each 128-column block with those rows' solution values is
// split into bwd_parts(rows) parts of bwd_part_rows(rows) rows (the last one
// shorter), each computed by its own CTA and published for the block's CTA,
// so that the rows stream on many SMs instead of one.  0: the block's CTA
// computes the product itself.  Part h of block b has backward key
// -1 - (b BWD_PARTS_MAX + h).
constexpr int BWD_PARTS_MAX = 8;
constexpr int BWD_PART_MIN_ROWS = 1024;
#if defined(__CUDACC__)
#define SGN_HD __host__ __device__
#else
#define SGN_HD
#endif
SGN_HD inline int bwd_part_rows(int64_t rows) {
  int64_t h = (rows + BWD_PART_MIN_ROWS - 1) / BWD_PART_MIN_ROWS;
  if (h > BWD_PARTS_MAX) h = BWD_PARTS_MAX;
  const int64_t rp = (rows + h - 1) / h;
  return (int)((rp + 127) / 128 * 128);
}
SGN_HD inline int bwd_parts(int64_t rows) {
  if (rows <= BWD_PART_MIN_ROWS) return 0;
  const int64_t rp = bwd_part_rows(rows);
  return (int)((rows + rp - 1) / rp);
}
#undef SGN_HD

// one CTA of an outer block's panel kernel: a 128-row band of front q (q
// indexes the level-ordered front list)
struct BandItem {
  int32_t q, band;
};

// one multifrontal store: fronts + pivots + solve buffers of one kind
struct Store {
  bool enabled = false;
  int dpn = 0;              // DOFs per node: 2d (saddle point) or d (K alone)
  bool kkt = true;          // saddle-point system (else K alone)
  bool fp32 = false;        // element type of the fronts
  void *F = nullptr;        // fronts, column-major f x f each
  void *W = nullptr;        // W = L21 D workspace, (f - K0) x FACTOR_BLOCK per front
  void *Ldg = nullptr;      // factored diagonal blocks staged by the panel kernel (panel per DOF)
  // FP32 fronts only: K-major copies of W and L21 of the current outer block,
  // split as hi (TF32-exact) + lo, rows = absolute front rows, for the
  // tensor-core trailing update; and one set of TMA tensor maps per front
  // two sets (outer blocks alternate between them, so that one block's
  // trailing update can still read its operands while the next block's
  // panels write theirs): wk[4 * parity + q], q = Whi, Wlo, Lhi, Llo
  float *wk[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  void *maps = nullptr;     // [2][n_sn] tensor maps, one set per parity
  bool tc = false;          // tensor-core trailing update available
  double *rhs = nullptr;    // per-front solve buffers (f each)
  double *yz = nullptr;     // per fully-summed DOF: y, then z = D^{-1} y, then v (solves)
  int32_t *piv_type = nullptr, *piv_perm = nullptr;  // per fully-summed DOF
  double *D0 = nullptr, *D1 = nullptr;
  // a front of order f with ns fully-summed columns keeps its first ns
  // columns (f x ns, the factor) at front_off, and its contribution block
  // (the (f - ns)^2 Schur complement handed to the parent) at cb_off in CB, an
  // arena shared by contribution blocks whose lifetimes (from their own
  // level's assembly to their parent's) do not overlap
  void *CB = nullptr;
  // inverses of the 128-wide unit-lower diagonal blocks of the factor, each
  // a dense row-major w x w block (X(j, i) at j * w + i), contiguous per front
  void *Xinv = nullptr;
  // dataflow substitutions: one CTA per 128-row band (forward) or 128-column
  // block (backward) of a front, listed per level in an order where every
  // band depends only on earlier entries; pub holds each published block
  // value (FP32 fronts: the value's bits with the solve's 32-bit tag in one
  // 64-bit word; FP64 fronts: the value, announced by the tag in pflag at the
  // block's first position); ctl = {solve counter, ticket, finished CTAs}
  unsigned long long *pub = nullptr;
  unsigned *pflag = nullptr, *ctl = nullptr;
  // FP32 fronts: the published parts of the backward ancestor-row products,
  // part h of front s's block at column k at bpart[part_off[s] + h ns + k + t]
  // (value bits and tag in one 64-bit word, as in pub; only fronts whose
  // product is split hold parts)
  unsigned long long *bpart = nullptr;
  const int64_t *part_off = nullptr;
  std::vector<int64_t> h_part_off;
  int64_t part_elems = 0;
  const SolveItem *fwd_items = nullptr, *bwd_items = nullptr;
  std::vector<SolveItem> h_fwd_items, h_bwd_items;
  std::vector<int64_t> h_fwd_lvl, h_bwd_lvl;  // per level: range in the item lists
  bool sched_ok = true;  // every item listed after the items it waits on
  // panel kernel of each (level, outer block): its bands, every front's
  // bands 0 and 1 (the panels' owners) first; fflag: two flags per pivot
  // position (used at each panel's first pivot), set to the factorization's
  // epoch (ctl[4]): [0, piv_elems) once the panel is factored, [piv_elems,
  // 2 piv_elems) once the panel's rows are final in the outer block's
  // earlier columns
  const BandItem *blk_items = nullptr;
  std::vector<BandItem> h_blk_items;
  std::vector<int64_t> h_blk_off;
  // tensor-core trailing update of each (level, outer block) b and tile
  // window w (0: the next block's FACTOR_BLOCK / 128 tile columns, 1: the
  // rest, 2: all): h_upd_off[3 b + w] = offset of its cumulative per-front
  // tile counts (active fronts + 1 entries) in upd_cum / h_upd_cum
  const int32_t *upd_cum = nullptr;
  std::vector<int32_t> h_upd_cum;
  std::vector<int64_t> h_upd_off;
  unsigned *fflag = nullptr;
  const int64_t *front_off = nullptr, *cb_off = nullptr, *w_off = nullptr, *rhs_off = nullptr, *piv_off = nullptr;
  const int64_t *xinv_off = nullptr;
  std::vector<int64_t> h_front_off, h_cb_off, h_w_off, h_rhs_off, h_piv_off, h_xinv_off;
  int64_t front_elems = 0, cb_elems = 0, w_elems = 0, rhs_elems = 0, piv_elems = 0, xinv_elems = 0;
  int64_t cb_sum = 0;  // sum of all contribution blocks (what the arena saves against)
  bool factored = false;
  // stabilization of the saddle-point fronts (eps_x on the x diagonal,
  // -eps_l on the lambda diagonal): 0 for the factor of the matrix itself
  double eps_x = 0.0, eps_l = 0.0;
  // CUDA graphs of the static launch sequences (captured once, replayed)
  cudaGraphExec_t fgraph = nullptr;        // factorization
  cudaGraphExec_t fgraph_prof = nullptr;   // factorization with events around the trailing updates
  std::vector<struct GraphEv> fprof;       // those events
  int64_t fgraph_launches = 0, fgraph_tc = 0;
  cudaGraphExec_t sgraph = nullptr;        // substitutions for one (b, x) pair
  const double *sgraph_b = nullptr;
  double *sgraph_x = nullptr;
  int64_t sgraph_launches = 0;
};

// an event pair recorded inside a captured graph (re-recorded on every replay)
struct GraphEv {
  int kind;
  double flops;
  cudaEvent_t e0, e1;
};

struct Ctx {
  Symbolic S;
  double E0 = 0.0, nu = 0.0;
  int stores = 0;
  cudaStream_t stream = nullptr;
  int device = -1;
  int num_sms = 152;
  int update_ctas = 0;              // CTAs per tensor-core trailing update (0: num_sms)
  bool bound = false;

  // carving
  char *base = nullptr;
  size_t bytes = 0;

  DevSym ds;
  // host copies needed for launches
  std::vector<int64_t> h_lvl_ptr;   // level -> offset into lvl_fronts
  std::vector<int64_t> h_item_ptr;  // level -> offset into items
  std::vector<std::vector<int32_t>> h_lvl_ns_nodes;  // per level: nown of each front in order

  // dynamic arrays
  int n_state = 0;                  // element state doubles per element
  double *st = nullptr;             // [n_state][n_elem]
  double *cpv = nullptr;            // [(d+1)*d][n_elem] element forces = columns of dc/dp
  double *Kv = nullptr, *Gv = nullptr;   // [nnzb][d*d]
  double *wA = nullptr, *tgt = nullptr;  // [n_x] tracked weight / target (rank-DOF layout)
  double *fx = nullptr, *fp = nullptr;   // df/dx [n_x], df/dp [n_elem] at the last assembly
  double *xr = nullptr;             // [n_x] positions at the last assembly (rank-DOF)
  double alpha = 0.0;
  double f_const = 0.0;             // 1/2 sum w t^2 lost when repeated tracked DOFs are merged
  double max_w = 0.0;               // largest |tracked weight|
  double res_eps_x = 0.0, res_eps_l = 0.0;  // regularization the residuals include (solves of M(delta))
  bool have_objective = false, assembled = false;
  double *lbq = nullptr, *lbr = nullptr;  // [n_elem] scratch of the L-BFGS two-loop recursion

  // refinement vectors (rank-DOF for x and lambda, element order for p)
  double *bx = nullptr, *bp = nullptr, *bl = nullptr;
  double *zx = nullptr, *zp = nullptr, *zl = nullptr;
  double *rx = nullptr, *rp = nullptr, *rl = nullptr;
  double *red = nullptr;            // reduced rhs / solution [n_free * 2d]
  static constexpr int KRY_VECS = 8;  // BiCGSTAB: r^, p, -v, y, s, z~, -t, zero
  double *kry = nullptr;            // [KRY_VECS][2 n_x + n_p]
  double *partial = nullptr;        // reduction scratch
  double *partial2 = nullptr;       // [2][n_partial]: ||r||^2, ||b||^2 partial sums of a graph step
  int n_partial = 0;
  int *status = nullptr;            // device status word
  int64_t *counters = nullptr;      // pivot counters (perturbed, 2x2, pos, neg, zero)
  double *eq = nullptr;             // equilibrium scratch: [4][n_x]
  double *xsave = nullptr, *xrt = nullptr;   // [n_nodes*d], [n_x]
  double *ueq = nullptr;            // Newton iterate u = x - X [n_nodes*d]
  double *hx = nullptr, *hdx = nullptr, *hdl = nullptr;  // host-call staging [n_nodes*d]
  double *hp = nullptr, *hdp = nullptr;                  // host-call staging [n_elem]

  // batched instances (sgn_batch_setup): instance i owns nodes
  // [inst_node_off[i], inst_node_off[i+1]) and elements likewise
  int n_inst = 0;
  std::vector<int64_t> inst_node_off, inst_elem_off;
  std::vector<int32_t> h_rank_inst, h_elem_inst;
  const int32_t *rank_inst = nullptr, *elem_inst = nullptr;  // device copies
  double *inst_acc = nullptr;       // [4][n_inst]: ||c||^2, ||f_ext||^2, ||r||^2, ||b||^2
  bool inst_have_eq = false, inst_have_kkt = false;
  bool pending_obj = false;         // objective given at set-up, applied at bind
  std::vector<int64_t> pobj_track;
  std::vector<double> pobj_target, pobj_weight;
  double pobj_alpha = 0.0;

  Store kkt64, kkt32, kf, kf32;
  Store *active = nullptr;          // saddle-point factor of the last sgn_factor

  std::string last_error;

  // measurement support
  int64_t launches = 0;
  int64_t tc_launches = 0;          // tensor-core trailing-update launches
  int prof_mask = 0;
  std::vector<cudaEvent_t> prof_ev; // pool; pairs (start, stop) in use order
  std::vector<int> prof_kind;       // kind of each used pair
  std::vector<double> prof_fl;      // flops of each used pair
  int64_t prof_used = 0;            // pairs used
  std::string prof_err;
  void count(int n = 1) { launches += n; }
  // event pair bracketing one launch of `kind` (nullptr if not profiled)
  cudaEvent_t *prof_pair(int kind, double flops = 0.0);
  // CUDA graphs
  bool use_graphs = true;
  cudaGraphExec_t step_graph = nullptr;    // sgn_step_graph
  const void *step_key[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int step_prec = -1, step_refine = -1;
  int64_t step_launches = 0, step_tc = 0;
  cudaStream_t cap_stream = nullptr;       // capture stream (the caller's may be the legacy stream)
  // a second stream for the part of each trailing update that the next
  // outer block's panels do not wait for, and the fork / join events
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::vector<GraphEv> *capture_events = nullptr;  // non-null while capturing a profiled graph
  std::vector<GraphEv> *pending_events = nullptr;  // events of the last profiled replay, not yet read
  double gacc_sec[8] = {0}, gacc_fl[8] = {0};
  int64_t gacc_n[8] = {0};
  void harvest_graph_events();
};

// brackets the launches issued in its scope with a profiled event pair
// (inside a graph capture the records become event-record nodes, so the pair
// can be timed after every replay of the graph)
struct ProfScope {
  Ctx &c;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ProfScope(Ctx &ctx, int kind, double flops = 0.0) : c(ctx) {
    if (cudaEvent_t *ev = ctx.prof_pair(kind, flops)) {
      e0 = ev[0];
      e1 = ev[1];
      record(e0);
    }
  }
  ~ProfScope() {
    if (e1) record(e1);
  }
  void record(cudaEvent_t e) {
    if (c.capture_events) cudaEventRecordWithFlags(e, c.stream, cudaEventRecordExternal);
    else cudaEventRecord(e, c.stream);
  }
};

// ---- launchers (assemble.cu)
void launch_elem_state(Ctx &c, const double *x, const double *p);       // at positions x
void launch_elem_state_disp(Ctx &c, const double *u, const double *p);  // at displacements u = x - X
void launch_slot_gather(Ctx &c, bool with_G);
void launch_elem_state_into(Ctx &c, const double *x, const double *p, double *st);
void launch_slot_gather_from(Ctx &c, const double *st);
void launch_objective_terms(Ctx &c, const double *x, const double *p);
void launch_reduce_rhs(Ctx &c, const double *bx, const double *bp, const double *bl, double *red, int dpn_kkt);
void launch_recover(Ctx &c, const double *red, const double *bp, double *zx, double *zp, double *zl);
void launch_residual(Ctx &c, const double *bx, const double *bp, const double *bl, const double *zx,
                     const double *zp, const double *zl, double *rx, double *rp, double *rl);
// r = b - K z over the free-rank DOFs (FP64, assembled K blocks)
void launch_residual_k(Ctx &c, const double *b, const double *z, double *r);
// returns sum of squares of the concatenation of (a, na), (b, nb), (c2, nc) on the host (synchronises)
double device_dot(Ctx &c, const double *a, const double *b, int64_t n);
// per-block partial sums of squares into partial_out (n_partial doubles), no synchronisation
void launch_sumsq3(Ctx &c, const double *a, int64_t na, const double *b, int64_t nb, const double *c2, int64_t nc,
                   double *partial_out);
double device_sumsq3(Ctx &c, const double *a, int64_t na, const double *b, int64_t nb, const double *c2, int64_t nc);
void launch_axpy(Ctx &c, double *y, const double *x, double a, int64_t n);
void launch_to_nodes(Ctx &c, const double *vr, double *out_nodes, double fixed_value_from_X);
void launch_to_nodes_plain(Ctx &c, const double *vr, double *out_nodes);
void launch_from_nodes(Ctx &c, const double *nodes, double *vr);
// equilibrium helpers
void launch_internal_force(Ctx &c, double *fr);      // f_int in rank-DOF layout from cpv
// disp: x holds displacements u = x - X (else positions)
void launch_energy_partials(Ctx &c, const double *x, const double *p, double *partials, int nblocks,
                            bool disp = false);
// out = v + s X over all node coordinates (node-major)
void launch_shift_rest(Ctx &c, const double *v, double s, double *out);
void launch_positions_update(Ctx &c, const double *x0, const double *dxr, double t, double *x);
int energy_blocks(Ctx &c);
void launch_gradient_finish(Ctx &c, const double *lam_r, double *g);

// ---- launchers (front.cu)
void factor_store(Ctx &c, Store &s);
void solve_store(Ctx &c, Store &s, const double *b_red, double *x_red);
void pivot_counts(Ctx &c, Store &s);  // fills c.counters (device)
void set_kernel_attributes();
void factor_direct(Ctx &c, Store &s);                                   // no graph
void wait_selftest(Ctx &c, Store &s);  // one substitution wait that must expire
cudaGraphExec_t capture_fn(Ctx &c, const std::function<void()> &body, int64_t *launches, int64_t *tc);
void solve_direct(Ctx &c, Store &s, const double *b_red, double *x_red);  // no graph
void destroy_graphs(Store &s);

// ---- batch.cu: per-instance norms of a batched handle (no-ops otherwise)
void batch_record_equilibrium(Ctx &c, const double *cr, const double *fr);
void batch_record_solve(Ctx &c);

// ---- lbfgs.cu: f(x, p) of the handle's objective (synchronises)
double objective_value(Ctx &c, const double *x, const double *p);

// ---- error reporting (api.cu): sets the handle's detail (if h) and the
// message sgn_strerror returns for the status
void set_error(Ctx *h, const std::string &msg);

// ---- static_scratch.cu: resolves the address of the library's fixed
// element-scratch array on `device` (current), once per device
cudaError_t static_scratch_bind(int device);

}  // namespace sgn

// the opaque handle of the C ABI is the context itself
struct sgn_ctx : public sgn::Ctx {};
