"""GB300-native differentiable Gaussian-splat rasterizer with a fast
gradient-accumulation backward (warp/SM/L2 reduction tiers)."""
