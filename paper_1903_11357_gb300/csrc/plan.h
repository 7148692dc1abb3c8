// Host-side plan of a preconditioner: partition, internal element order, tile envelopes of the
// local factors, Cholesky task lists, element groups and coarse agglomerate lists.
#pragma once

#include <vector>

#include "common.h"

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
  // backward stream: position b (subdomain s occupies the same index range as its forward tiles) holds
  // the tile bwd_src[b]; per subdomain, column J from the last: tiles (I, J), I > J, then (J, J)
  std::vector<long long> bwd_src;
  long long ntiles = 0;
  int max_nbt = 0;
  // Cholesky tasks, grouped by step K: diag (s, K), panel (s, I), update (s, I, J), I >= J
  std::vector<int> diag_off, panel_off, upd_off;  // [max_nbt + 1]
  std::vector<int> diag_task;   // s
  std::vector<int> panel_task;  // pairs (s, I)
  std::vector<int> upd_task;    // triples (s, I, J)
  // build from the first-column function of each subdomain's dof rows
  void build(const std::vector<std::vector<int>>& first_col);
};

struct Plan {
  int ne = 0, np = 0, nsub = 0, nagg = 0, q = 0, nq = 0;
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

int build_plan(const dgasm_system_s& sys, int nsub, int ncoarse, int q, const int* sub_in, const int* agg_in, Plan& P);

}  // namespace dgasm
