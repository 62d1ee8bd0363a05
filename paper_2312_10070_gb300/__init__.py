"""GB300-native differentiable 3D-Gaussian rasterizer of Gaussian-SLAM (arXiv 2312.10070)."""
