// Register line-FFT plans for grid sizes 128-144 (kernels in fft_reg.cuh).
#include "fft_reg.cuh"

extern const pw_reg_plan pw_reg_plans_d[] = {
    PW_REG_PLAN(32, 4), PW_REG_PLAN(16, 8),
    PW_REG_PLAN(16, 9),
};
extern const int pw_reg_nplans_d = sizeof(pw_reg_plans_d) / sizeof(pw_reg_plans_d[0]);
