// Host-side symbolic analysis: geometric nested dissection, interfaces and the
// clustering hierarchy (Section 2.2, Fig. 2-3; merging, Section 2.6).
//
// Readings for structured grids (the paper gives the scheme only by figures):
//  * complete binary tree of depth L in heap numbering; a node cuts its
//    longest box axis (ties to the lowest axis) at mid = (lo + hi) / 2; the
//    separator is the plane v[axis] = mid, children [lo, mid) and [mid+1, hi);
//    leaves (level L) keep their whole box;
//  * at stage k a separator S is split into interfaces by the key
//    {(D, sign(v[axis_D] - mid_D))} over descendants D of S with
//    level(S) < level(D) < k, axis_D != axis_S, whose box widened by one on
//    every side contains v; equal keys form one interface;
//  * clusters of a stage are ordered by (node id, key) with lexicographic key
//    order; merging to stage k-1 drops the pairs of level k-1.
#pragma once
#include <cstdint>
#include <utility>
#include <vector>

namespace spaqr {

struct NdNode {
  int id = 0, level = 0;
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  int axis = -1, mid = -1;
  bool empty = true;
  std::vector<int32_t> verts;  // ascending
};

struct StageClusters {
  int stage = 0;
  std::vector<int32_t> node, level;
  std::vector<int64_t> vptr;      // vertex lists (CSR), ascending ids per cluster
  std::vector<int32_t> verts;
  std::vector<int32_t> parent;    // id at stage-1, -1 when eliminated at this stage
};

struct Analysis {
  int nx = 0, ny = 0, nz = 0, depth = 0;
  int64_t n = 0;
  double seconds = 0.0;
  std::vector<NdNode> nodes;
  std::vector<StageClusters> stages;  // stages[k] for k = 1..depth (index 0 unused)
};

// Builds the full analysis; throws std::invalid_argument on bad sizes.
Analysis* build_analysis(int nx, int ny, int nz, int depth);
// The same structure from graph(A^T A) of a CSR matrix (symbolic_alg.cpp):
// algebraic nested dissection, interfaces by adjacency, merge hierarchy.
Analysis* build_analysis_matrix(int64_t m, int64_t n, const int64_t* rowptr, const int32_t* colidx, int depth);
// Maximum-weight column-perfect row matching (sum of log|a_ij|); false if none exists.
bool max_weight_matching(int64_t m, int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* vals,
                         int32_t* match);

}  // namespace spaqr
