// Binomial recompute-checkpointing plan (Griewank & Walther, "revolve"), the
// memory-bounded way to give the adjoint its forward history in reverse order (Sec. 1:
// keep a few states, recompute the rest from the nearest stored one).
//
// Model: the adjoint of step n needs forward state n; the zero initial state is always
// available; `s` slots can each hold one state; the first forward pass also runs the
// last step (nt-1 -> nt) for its receiver record.  The plan is the optimal recursion
//
//   T(l, s) = min_j [ j + T(l - j, s - 1) + T(j, s) ],  T(1, s) = 0,  T(l, 0) = l(l-1)/2
//
// (advance j steps and store that state, reverse the right part with one slot fewer,
// restore, reverse the left part), evaluated with its closed form
//   T(l, s) = r l - beta(s + 2, r - 1),  beta(S, r) = C(S + r, S),
//   r = min { r : beta(s + 1, r) >= l }.
#include <vector>

#include "aew_revolve.h"

namespace aew {

static long long binom_capped(int S, int r, long long cap) {
  // C(S + r, r), saturating at cap + 1
  if (r < 0) return 0;
  long double b = 1.0L;
  for (int i = 1; i <= r; ++i) {
    b = b * (long double)(S + i) / (long double)i;
    if (b > (long double)cap) return cap + 1;
  }
  return (long long)(b + 0.5L);
}

long long revolve_cost(long long l, int s) {
  if (l <= 1) return 0;
  if (s <= 0) return l * (l - 1) / 2;
  const int S = s + 1;
  int r = 0;
  while (binom_capped(S, r, l) < l) ++r;
  const long long big = (long long)4e18;
  return (long long)r * l - binom_capped(S + 1, r - 1, big);
}

namespace {

struct Planner {
  std::vector<RevAction>& out;
  int nt;
  int s_total;
  bool final_done = false;
  long long fwd = 0;

  void emit(int op, int arg) { out.push_back(RevAction{op, arg}); }
  void reverse_one(int n) {
    if (n == nt - 1 && !final_done) {
      emit(kOpFinal, nt - 1);
      final_done = true;
      ++fwd;
    }
    emit(kOpReverse, n);
  }
  // precondition: the live state is `a`, restorable from slot_a (-1: zero state)
  void range(int a, int l, int s_free, int slot_a) {
    if (l == 1) {
      reverse_one(a);
      return;
    }
    if (s_free == 0) {
      for (int n = a + l - 1; n >= a; --n) {
        if (n != a + l - 1) emit(kOpRestore, slot_a);
        if (n > a) {
          emit(kOpAdvance, n - a);
          fwd += n - a;
        }
        reverse_one(n);
      }
      return;
    }
    long long best = -1;
    int bj = 1;
    for (int j = 1; j < l; ++j) {
      const long long c = j + revolve_cost(l - j, s_free - 1) + revolve_cost(j, s_free);
      if (best < 0 || c <= best) {
        best = c;
        bj = j;
      }
    }
    const int slot = s_total - s_free;
    emit(kOpAdvance, bj);
    fwd += bj;
    emit(kOpStore, slot);
    range(a + bj, l - bj, s_free - 1, slot);
    emit(kOpRestore, slot_a);
    range(a, bj, s_free, slot_a);
  }
};

}  // namespace

long long revolve_plan(int nt, int s, std::vector<RevAction>& out) {
  out.clear();
  if (nt < 1 || s < 0) return -1;
  Planner p{out, nt, s};
  p.range(0, nt, s, -1);
  return p.fwd;
}

}  // namespace aew
