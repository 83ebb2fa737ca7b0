// Register line-FFT plans for grid sizes 48-72 (kernels in fft_reg.cuh).
#include "fft_reg.cuh"

extern const pw_reg_plan pw_reg_plans_b[] = {
    PW_REG_PLAN(16, 3), PW_REG_PLAN(8, 6), PW_REG_PLAN(4, 12),
    PW_REG_PLAN(32, 2), PW_REG_PLAN(16, 4), PW_REG_PLAN(8, 8),
    PW_REG_PLAN(8, 9),
};
extern const int pw_reg_nplans_b = sizeof(pw_reg_plans_b) / sizeof(pw_reg_plans_b[0]);
