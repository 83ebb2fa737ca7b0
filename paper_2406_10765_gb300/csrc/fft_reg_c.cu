// Register line-FFT plans for grid size 96 (kernels in fft_reg.cuh).
#include "fft_reg.cuh"

extern const pw_reg_plan pw_reg_plans_c[] = {
    PW_REG_PLAN(32, 3), PW_REG_PLAN(16, 6), PW_REG_PLAN(8, 12),
};
extern const int pw_reg_nplans_c = sizeof(pw_reg_plans_c) / sizeof(pw_reg_plans_c[0]);
