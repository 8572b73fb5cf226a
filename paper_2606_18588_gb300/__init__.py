"""GB300-native pixel-level local rendering and global composition for 3D Gaussian
Splatting (Splaxel): K Gaussian subsets rendered to partial pixel images, composited in
per-pixel depth order, differentiated and optimised with Adam, all in hand-written CUDA
for sm_103a behind a C-ABI library (libsplx.so)."""
