// Host-side binomial checkpointing planner (see aew_revolve.cpp).
#pragma once

#include <vector>

namespace aew {

enum { kOpAdvance = 0, kOpStore = 1, kOpRestore = 2, kOpFinal = 3, kOpReverse = 4 };

struct RevAction {
  int op;
  int arg;
};

// Minimal forward steps to reverse l steps with s free slots (first state available).
long long revolve_cost(long long l, int s);

// Full action list for a gradient over nt steps with s slots; returns the number of
// forward steps of the plan (revolve_cost(nt, s) + 1), or -1 for bad arguments.
long long revolve_plan(int nt, int s, std::vector<RevAction>& out);

}  // namespace aew
