// Host-side plan of a preconditioner: partition, internal element order, tile envelopes of the
// local factors, Cholesky task lists, element groups and coarse agglomerate lists.
#pragma once

#include <vector>

#include "common.h"
#include "engine.h"

namespace dgasm {

constexpr int TILE = 32;  // tile edge of the local Cholesky factors

void rcb_parts(const MeshData& m, std::vector<int> elems, int k, std::vector<int>& part_of, int first_part);
int compute_partition(const MeshData& m, int nsub, int ncoarse, std::vector<int>& sub, std::vector<int>* agg);

// Tile-envelope structure of a set of dense lower-triangular factors ("subdomains").  Tile row I of
// subdomain s holds tiles (I, F(I)) .. (I, I), stored contiguously from tile index trow_ptr.
struct Envelope {
  int nsub = 0;
  std::vector<int> ndof;               // [nsub] dofs per subdomain
  std::vector<int> sub_trow;           // [nsub+1] offsets into the tile-row arrays
  std::vector<int> trow_F;             // first tile column of each tile row
  std::vector<long long> trow_ptr;     // tile index of the first tile of each tile row
  long long ntiles = 0;
  // Super-rows: groups of sr consecutive tile rows.  The triangular solves use, per super-row q, the
  // explicit inverse X_q of its lower-triangular diagonal block (ntr(ntr+1)/2 tiles, ntr <= sr, row-major
  // tile order (i, j), j <= i), and the factor tiles that couple different super-rows.
  std::vector<int> sub_sr;               // [nsub+1] first global super-row of each subdomain
  std::vector<long long> dinv_ptr;       // [nsr+1] first tile of each super-row's inverse block
  long long ndinv = 0;
  // Streams in the order the sweeps consume them, made of runs: a run is a sequence of tiles that all
  // add into one output block, with consecutive operand blocks.  Per super-row q, runs o = 0..ntr-1:
  //   forward:  coupling run o = tiles (I0+o, J), J = F .. I0-1 (operand y_J), then
  //             inverse run o = X_q tiles (o, j), j = 0..o (operand t_j);
  //   backward (super-rows descending): coupling run o = tiles (I, I0+o), I = first .. last tile row
  //             below the super-row with F(I) <= I0+o (operand x_I; a zero tile where a row in between
  //             does not reach column I0+o), then inverse run o = X_q tiles (i, o), i = o..ntr-1.
  // Entry >= 0 is a factor tile index, ZERO_TILE a tile of zeros, other entries < 0 are
  // -(inverse-block tile index + 1).
  std::vector<long long> fwd_ptr, bwd_ptr;   // [nsub+1] each subdomain's range in each stream
  std::vector<long long> fwd_src, bwd_src;
  std::vector<int> dinv_task;            // per super-row: (subdomain, first tile row, tile rows)
  // coupling runs: [global super-row][sr][2] = (first operand block, tiles)
  std::vector<int> fwd_run, bwd_run;
  int max_nbt = 0;
  // Cholesky tasks, grouped by step K: diag (s, K), panel (s, I), update (s, I, J), I >= J
  std::vector<int> diag_off, panel_off, upd_off;  // [max_nbt + 1]
  std::vector<int> diag_task;   // s
  std::vector<int> panel_task;  // pairs (s, I)
  std::vector<int> upd_task;    // triples (s, I, J)
  // the same updates grouped for the tensor-core kernel: per (s, K) the panel P = [L_IK], I in S(s, K)
  // (n tiles, panel_task entries pstart .. pstart+n-1) and C_IJ -= (P P^T)_IJ, I >= J, cut into blocks of
  // 4 row tiles (mb) x 8 column tiles (nb): quadruples (pstart, n, mb, nb)
  std::vector<int> tc_off;      // [max_nbt + 1]
  std::vector<int> tc_task;
  int sr = 4;                            // tile rows per super-row
  // build from the first-column function of each subdomain's dof rows, with super-rows of sr_ tile rows
  void build(const std::vector<std::vector<int>>& first_col, int sr_);
};

// R_0^T of a non-nested coarse mesh in internal element order: pairs (element i, coarse cell J) with blocks
// [np][nq] (row a, column c), grouped by element (ptr, ascending J) and listed again by coarse cell (tptr,
// tpair: pair indices, ascending)
struct R0TPairs {
  std::vector<int> ptr, col, elem, tptr, tpair;
  std::vector<double> blocks;
};
int nonnested_r0t(const MeshData& fine, const std::vector<int>& perm, const MeshData& coarse, int p, int q,
                  R0TPairs& out);

struct Plan {
  int ne = 0, np = 0, nsub = 0, nagg = 0, q = 0, nq = 0;
  bool nonnested = false;            // coarse space on an independent mesh (nagg = its cell count)
  std::vector<int> sub_of, agg_of;   // caller's element order
  std::vector<int> perm, iperm;      // perm[internal] = caller element; iperm inverse
  std::vector<int> sub_e0;           // [nsub+1] internal element ranges
  // matrix in internal order
  std::vector<int> rowptr, col;
  std::vector<long long> src_blk;    // source block (caller order CSR) of each internal block
  Envelope env;                      // local factors
  // element groups for the fused update/restriction kernel: agglomerates, or chunks of elements
  std::vector<int> grp_ptr, grp_elems;
  int ngrp = 0;
  std::vector<int> agg_int;          // agglomerate of each internal element (or -1)
  std::vector<double> agg_bbox;      // [nagg * 4]
  Envelope env0;                     // coarse factor (one dense block)
};

// sr: tile rows per super-row of the local factors (the coarse factor takes super_row(DGASM_FP64))
// coarse: an independent coarse mesh (non-nested coarse space); ncoarse and agg_in are then ignored
int build_plan(const dgasm_system_s& sys, int nsub, int ncoarse, int q, const int* sub_in, const int* agg_in, int sr,
               Plan& P, const MeshData* coarse = nullptr);

}  // namespace dgasm
