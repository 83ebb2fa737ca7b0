// Register line-FFT plans for grid sizes 16-36 (kernels in fft_reg.cuh).
#include "fft_reg.cuh"

extern const pw_reg_plan pw_reg_plans_a[] = {
    PW_REG_PLAN(16, 1), PW_REG_PLAN(8, 2), PW_REG_PLAN(4, 4),
    PW_REG_PLAN(8, 3), PW_REG_PLAN(4, 6),
    PW_REG_PLAN(32, 1), PW_REG_PLAN(16, 2), PW_REG_PLAN(8, 4),
    PW_REG_PLAN(4, 9),
};
extern const int pw_reg_nplans_a = sizeof(pw_reg_plans_a) / sizeof(pw_reg_plans_a[0]);
