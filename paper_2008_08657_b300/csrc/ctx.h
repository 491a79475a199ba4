// Definition of the opaque lmfao_ctx handle of include/lmfao.h (shared by the host files).
#pragma once

#include "plan.h"

// The root relation reorganised into segment order for one segment key, kept across plans so
// that a new batch over the same relations (every level of a decision tree, for instance) does
// not sort the root relation again. Owned by the context.
struct lmfao_reorg {
  int root = -1;
  std::vector<int> segcols;
  std::vector<int64_t> hist;        // tuples per segment
  unsigned int *dest = nullptr;     // device: row -> position in segment order
  std::map<int, void *> cols;       // root column -> device copy in segment order (+16 bytes)
};

// One physical plan of a batch whose queries need different roots: the plan, its join tree and
// the batch's query ids it evaluates (its local query i is batch query qids[i]).
struct lmfao_subplan {
  lmfao::PhysPlan *plan = nullptr;
  lmfao::JoinTree tree;
  std::vector<int> qids;
};

struct lmfao_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;  // internal stream for loading and planning
  std::string last_error;
  std::vector<lmfao::Relation> rels;
  std::vector<lmfao::QueryIn> queries;
  lmfao::JoinTree tree;
  lmfao::LogicalPlan logical;
  lmfao::PhysPlan *plan = nullptr;
  bool planned = false, ran = false;
  cudaStream_t run_stream = nullptr;
  // fetch buffers
  std::vector<int32_t> fk;
  std::vector<int64_t> fc;
  std::vector<double> fs;
  // profiling
  bool profiling = false;
  std::vector<cudaEvent_t> events;
  std::vector<std::string> ev_names;
  std::vector<std::string> kernel_names;
  std::vector<lmfao_reorg> reorg;   // reorganised root relations (see lmfao_reorg)
  // side streams on which the views of different subtrees of the root run concurrently (created
  // when a plan first has views in two subtrees; fork / join events)
  static constexpr int kViewLanes = 4;
  cudaStream_t view_stream[kViewLanes] = {};
  cudaEvent_t view_fork = nullptr, view_join[kViewLanes] = {};
  // A batch planned with several physical roots (plan == nullptr then): one plan per root.
  std::vector<lmfao_subplan> subs;
  std::vector<std::pair<int, int>> qroute;  // batch query -> (index in subs, local query id)
};
