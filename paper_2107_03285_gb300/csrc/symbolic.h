// Host symbolic phase of the SGN saddle-point factorization.
//
// The sparsity of Eq. sparseSystemGN is fixed by the mesh (Sec. 4), so this
// runs once per mesh on the host and its result is reused by every
// assemble / factor / solve.  Everything here works on the graph of free
// nodes: two free nodes are adjacent when an element contains both.
//
// Unknown layout of the reduced (p-eliminated) saddle-point system: a free
// node of elimination rank r owns the 2d DOFs
//     r*2d + 2a + 0 = x_{r,a},   r*2d + 2a + 1 = lambda_{r,a},   a < d,
// i.e. every state DOF sits next to its multiplier.  Any set of such
// (x, lambda) pairs gives a nonsingular principal submatrix
// [[A_SS, K_SS], [K_SS, -G_SS]] (K SPD, A and G = cp C^{-1} cp^T PSD), which
// is what lets Bunch-Kaufman pivoting stay inside each panel of even width.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace sgn {

struct SymbolicOptions {
  int leaf_nodes = 16;
  int panel = 32;
};

struct Supernode {
  int first = 0;          // first elimination rank of its own nodes
  int nown = 0;           // own nodes (ranks first .. first+nown-1)
  int nstruct = 0;        // nodes below the diagonal block
  int64_t struct_off = 0; // into Symbolic::struct_ranks / relpos
  int parent = -1;        // elimination-tree parent (-1: root)
  int level = 0;          // 0 for leaves, 1 + max(children) otherwise
  int child_off = 0;      // into Symbolic::children
  int nchild = 0;
  int fnodes() const { return nown + nstruct; }
};

struct Symbolic {
  int dim = 0;
  int n_nodes = 0, n_elem = 0, n_free = 0;
  SymbolicOptions opts;

  // node numbering
  std::vector<int32_t> node_rank;   // [n_nodes] elimination rank, -1 if fixed
  std::vector<int32_t> rank_node;   // [n_free]

  // element data (SoA over elements)
  std::vector<int32_t> elem_node;   // [(d+1) * n_elem] node ids, [a*n_elem + e]
  std::vector<int32_t> elem_rank;   // [(d+1) * n_elem] ranks, -1 if fixed
  std::vector<double> elem_B;       // [(d+1)*d * n_elem] shape gradients, [(a*d+j)*n_elem + e]
  std::vector<double> elem_vol;     // [n_elem]
  std::vector<double> X;            // [n_nodes * d] rest positions (node-major)

  // block pattern of K over ranks: full symmetric block CSR, diagonal included
  std::vector<int32_t> bsr_ptr;     // [n_free + 1]
  std::vector<int32_t> bsr_col;     // [nnzb] sorted ranks
  std::vector<int32_t> bsr_diag;    // [n_free] slot of (r, r)
  std::vector<int32_t> bsr_orig_pos;// [nnzb] front node position of the column (c >= r) in owner(r)'s front, else -1

  // gather map: for each upper slot (r <= c) its contributions (e, a, b)
  std::vector<int32_t> up_slot;     // [n_up] slot of (r, c)
  std::vector<int32_t> up_slot_t;   // [n_up] slot of (c, r)
  std::vector<int32_t> up_ptr;      // [n_up + 1]
  std::vector<int32_t> up_contrib;  // packed e*16 + a*4 + b

  // node -> incident elements (free nodes), packed e*4 + a
  std::vector<int32_t> inc_ptr;     // [n_free + 1]
  std::vector<int32_t> inc;

  // supernodes in postorder (children before parents)
  std::vector<Supernode> sn;
  std::vector<int32_t> struct_ranks;   // concatenated struct lists (sorted ranks)
  std::vector<int32_t> relpos;         // position of each struct node in the parent's front
  std::vector<int32_t> children;       // concatenated child lists
  std::vector<int64_t> cmap_off;       // per child entry: offset into cmap
  std::vector<int32_t> cmap;           // for (parent s, child j): per parent front node P the child's struct index, -1 if none
  std::vector<int32_t> sn_of_rank;     // [n_free]
  int n_levels = 0;
  std::vector<std::vector<int32_t>> level_fronts;  // per level, sorted by nown descending

  // statistics for the reduced saddle-point system (2d DOFs per node) and K alone
  int64_t max_front_nodes = 0;
  int64_t nnz_factor_kkt = 0;
  double flops_kkt = 0.0, flops_k = 0.0;
  int64_t sum_f2_nodes = 0;            // sum over fronts of fnodes^2
  double seconds = 0.0;
};

// Builds the symbolic structure.  Returns an empty string on success, else a
// message describing the invalid input.
std::string analyze(int dim, int n_nodes, int n_elem, const double *X, const int32_t *conn,
                    const uint8_t *fixed, const SymbolicOptions &opts, Symbolic &out);

}  // namespace sgn
