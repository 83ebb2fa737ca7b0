// FFT plans of the local part of H psi: the register line-FFT plans of the
// fft_reg_*.cu units in one table, and the plan a cell uses per precision.
#include "pw_internal.cuh"

extern const pw_reg_plan pw_reg_plans_a[], pw_reg_plans_b[], pw_reg_plans_c[], pw_reg_plans_d[];
extern const int pw_reg_nplans_a, pw_reg_nplans_b, pw_reg_nplans_c, pw_reg_nplans_d;

namespace {

struct PlanTable {
  const pw_reg_plan *p;
  const int *n;
};
const PlanTable kTables[] = {{pw_reg_plans_a, &pw_reg_nplans_a},
                             {pw_reg_plans_b, &pw_reg_nplans_b},
                             {pw_reg_plans_c, &pw_reg_nplans_c},
                             {pw_reg_plans_d, &pw_reg_nplans_d}};

constexpr size_t kDefaultBatchBytes = (size_t)64 << 20;   // z-pencils of a batch stay in L2

}  // namespace

int pw_reg_plan_count() {
  int n = 0;
  for (const PlanTable &t : kTables) n += *t.n;
  return n;
}

const pw_reg_plan *pw_reg_plan_at(int i) {
  if (i < 0) return nullptr;
  for (const PlanTable &t : kTables) {
    if (i < *t.n) return &t.p[i];
    i -= *t.n;
  }
  return nullptr;
}

bool pw_reg_plan_fits(const pw_cell *c, int i, int fp32, int compact) {
  const pw_reg_plan *p = pw_reg_plan_at(i);
  if (!p) return false;
  const int n = c->N[0];
  if (c->N[1] != n || c->N[2] != n || p->N != n) return false;
  // the y-columns that meet the sphere must not wrap onto each other
  if (2 * c->mxmax + 1 > n) return false;
  return p->smem(c, fp32, compact) <= 227 * 1024;   // plane in shared memory
}

namespace {
// default: the first plan listed for the grid size with the full plane,
// else the first with the compact plane; (-1, 0) for the Stockham passes
void default_plan(const pw_cell *c, int fp32, int *plan, int *compact) {
  const int np = pw_reg_plan_count();
  for (int cp = 0; cp < 2; ++cp)
    for (int i = 0; i < np; ++i)
      if (pw_reg_plan_fits(c, i, fp32, cp)) { *plan = i; *compact = cp; return; }
  *plan = -1;
  *compact = 0;
}
}  // namespace

int pw_cell_fft_plan(const pw_cell *c, int fp32) {
  const int chosen = c->fft_plan[fp32 ? 1 : 0];
  if (chosen >= -1) return chosen;
  int p, cp;
  default_plan(c, fp32, &p, &cp);
  return p;
}

int pw_cell_fft_compact(const pw_cell *c, int fp32) {
  if (c->fft_plan[fp32 ? 1 : 0] >= -1) return c->fft_compact[fp32 ? 1 : 0];
  int p, cp;
  default_plan(c, fp32, &p, &cp);
  return cp;
}

size_t pw_cell_fft_batch_bytes(const pw_cell *c, int fp32) {
  const size_t b = c->fft_batch[fp32 ? 1 : 0];
  return b ? b : kDefaultBatchBytes;
}
