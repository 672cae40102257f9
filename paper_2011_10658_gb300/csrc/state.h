// Definitions of the opaque C-ABI handles (shared by the C-ABI sources).
#pragma once
#include <vector>

#include "engine.h"
#include "model.h"

struct qed_model {
  qed::Params p;
  std::vector<qed::Term> terms;
  double constant = 0.0;
  std::vector<qed::TreeNode> nodes;
};

struct ttn_state {
  qed::Engine* engine = nullptr;
  const qed_model* model = nullptr;
};

// Sets the message returned by qed_last_error() on this thread.
void qed_set_last_error(const char* msg);
