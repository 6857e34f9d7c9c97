"""CPU oracle for the differentiable render-and-compare step.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the bench's
CPU-baseline leg may import or run anything in this package; the product path
never does. It shares no code with the CUDA path: the two meet only in the
seeded inputs from `synth`.

Layout:
  raster.c / visibility.py  float32 + int64 visibility (bit-exact contract)
  render.py                 float64 mesh frame, interpolation, mip-mapped
                            texture, shading, antialiasing, loss, Laplacian,
                            lambda schedule, Adam; gradients by reverse-mode
                            differentiation of that float64 forward with
                            visibility and texture LOD held fixed
  tessellate.py             edge-midpoint tessellation + displacement

Parity unpinned: the end-to-end optimization result (a simplified asset) is
not unique; only the single step is pinned.
"""
