// Internal interface between the U-Net and the solver (the public one is in wbfbt.h).
#pragma once

#include <cuda_runtime.h>

struct wbfbt_net;

// y = net(x) for one sample: x [n^3][cin], y [n^3][cout], FP32 device arrays, issued on st.
int unet_forward_into(wbfbt_net* net, const float* x, float* y, cudaStream_t st);
int unet_grid(const wbfbt_net* net);
int unet_channels_in(const wbfbt_net* net);
int unet_channels_out(const wbfbt_net* net);
