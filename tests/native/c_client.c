/*
 * A plain C99 client of the library: it includes only include/mpa.h, links
 * libmpa.so and uses the entry points that need no GPU (plan creation and
 * validation, workspace sizes, the scale check, split selection, status
 * strings).  It shows that the boundary is usable without C++ or Python;
 * tests/test_c_client.py builds and runs it.  A GPU run would go on with
 * cudaMalloc of the workspace, mpa_plan_set_workspace, mpa_plan_autotune
 * and mpa_propagate on a device field.
 */
#include <stdio.h>
#include <string.h>

#include "mpa.h"

static int failures = 0, checks = 0;

#define EXPECT(cond, what)                                             \
    do {                                                               \
        checks++;                                                      \
        if (!(cond)) {                                                 \
            fprintf(stderr, "FAIL line %d: %s\n", __LINE__, what);     \
            failures++;                                                \
        }                                                              \
    } while (0)

int main(void) {
    /* one DM span: 45 km of anomalous fiber, 5 km of compensating fiber */
    const mpa_segment span[2] = {
        {45.0, -21.7, 0.1, 1.3, 0.0},
        {5.0, 190.0, 0.1, 1.3, 0.0},
    };
    mpa_fiber_map map;
    memset(&map, 0, sizeof map);
    map.segments = span;
    map.n_segments = 2;
    map.gamma_per_km = mpa_gamma_from_db_per_km(0.2);
    map.z_a_km = 50.0;
    map.n_periods = 40;

    mpa_plan_params prm;
    memset(&prm, 0, sizeof prm);
    prm.N = (int64_t)1 << 20;
    prm.T_ps = 102400.0;
    prm.L_km = 5.0;
    prm.M = 125;
    prm.n_iter = 2;
    prm.precision = MPA_FP32;
    prm.schedule = MPA_SCHEDULE_AUTO;

    mpa_plan* plan = NULL;
    EXPECT(mpa_plan_create(&map, &prm, &plan) == MPA_OK && plan != NULL, "plan of the 2^20 link");

    size_t ws = 0;
    EXPECT(mpa_plan_workspace_size(plan, &ws) == MPA_OK, "workspace size");
    /* (M + 1) node spectra, their work copies, the FP64 state and the tables */
    EXPECT(ws >= (size_t)2 * 126 * ((size_t)1 << 20) * 8, "workspace holds the node spectra");

    double z_nl = 0.0, z_disp = 0.0;
    int32_t flags = -1;
    EXPECT(mpa_plan_check_scales(plan, 2e-3, 18.0, &z_nl, &z_disp, &flags) == MPA_OK, "weakly nonlinear scales");
    EXPECT(flags == 0 && z_nl > 300.0 && z_disp > 5.0, "z_nl and z_disp of the benchmark link");
    EXPECT(mpa_plan_check_scales(plan, 1.0, 18.0, NULL, NULL, &flags) == MPA_ERR_SCALES, "1 W is not weak");

    EXPECT(mpa_plan_set_split(plan, 10) == MPA_OK, "square split");
    EXPECT(mpa_plan_set_split(plan, 1) == MPA_ERR_UNSUPPORTED_N, "2-point columns refused");
    int32_t nseg = 0;
    EXPECT(mpa_plan_n_segments(plan, &nseg) == MPA_OK && nseg == 80, "physical segments");
    /* propagation without a workspace is refused before any CUDA call */
    EXPECT(mpa_propagate(plan, (void*)256, 0.0, 5.0, NULL) == MPA_ERR_WORKSPACE, "no workspace");
    mpa_plan_destroy(plan);

    prm.L_km = 7.0; /* neither divides nor is a multiple of the 50-km period */
    plan = NULL;
    EXPECT(mpa_plan_create(&map, &prm, &plan) == MPA_ERR_GRID && plan == NULL, "inconsistent grid");

    size_t ss = 0;
    EXPECT(ss_workspace_size((int64_t)1 << 20, MPA_FP64, &ss) == MPA_OK && ss == ((size_t)1 << 20) * 16,
           "split-step workspace");
    EXPECT(strcmp(mpa_status_string(MPA_ERR_GRID), "z-grid inconsistent with the fiber map") == 0, "status string");
    EXPECT(map.gamma_per_km > 0.0230258509299 && map.gamma_per_km < 0.0230258509300, "0.2 dB/km as gamma");

    if (failures) return 1;
    printf("C client: %d checks passed\n", checks);
    return 0;
}
