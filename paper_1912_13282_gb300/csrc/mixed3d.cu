// FP32 + refinement weights kernels for 3D stencils (see mixed_launch.cuh).
#include "mixed_launch.cuh"

int mixed_init_device_3d(mm_ctx *ctx) { return mixed_init(ctx); }

int mixed_launch_3d(mm_ctx *ctx, const WeightsJob &job, int *fb_count, int *fb_list) {
    return mixed_launch<3>(ctx, job, fb_count, fb_list);
}
