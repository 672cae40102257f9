// Batched sweeps of independent TTN problems (see batch.cu).
#pragma once

#include <map>
#include <memory>
#include <vector>

namespace qed {

class Engine;
struct SweepStats;

class BatchRunner {
 public:
  // Engines of the same lattice and precision, all on one CUDA stream.
  explicit BatchRunner(std::vector<Engine*> es);
  ~BatchRunner();
  // One sweep of every problem; stats accumulate per problem.
  int sweep(double tol, int max_krylov, std::vector<SweepStats>* stats);
  void set_graphs(bool on) { use_graphs_ = on; }

 private:
  struct Grouped;
  std::vector<Engine*> es_;
  std::map<int, std::unique_ptr<Grouped>> cur_;   // grouped product plan per node
  bool use_graphs_ = true;
  int build(int node, const std::vector<int>& members, std::unique_ptr<Grouped>* out);
  bool stale(const Grouped& g) const;
  int launch(Grouped& g);
  int product(int node, const std::vector<int>& active);
  int lanczos(int node, const std::vector<double>& tol, int max_krylov, bool mixed, int max_restarts,
              std::vector<double>* energy, std::vector<double>* resid, std::vector<int>* iters);
  int optimize(int node, double tol, int max_krylov, std::vector<SweepStats>* stats);
};

}  // namespace qed
