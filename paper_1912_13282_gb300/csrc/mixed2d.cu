// FP32 + refinement weights kernels for 2D stencils (see mixed_launch.cuh).
#include "mixed_launch.cuh"

int mixed_init_device_2d(mm_ctx *ctx) { return mixed_init(ctx); }

int mixed_launch_2d(mm_ctx *ctx, const WeightsJob &job, int *fb_count, int *fb_list) {
    return mixed_launch<2>(ctx, job, fb_count, fb_list);
}
