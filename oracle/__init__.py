"""CPU oracle for the active-set splatting hot path. TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package. The product path (the CUDA library and its Python binding) never
imports it and fails loudly when the CUDA library is missing. The oracle shares
no code, constants or helpers with the CUDA path; both consume the same seeded
inputs from `paper_2506_21117_gb300.synthetic`, which holds none of the
method's arithmetic.

What it computes, and where each part comes from:
  * fp32_index  - every quantity that decides an integer (tile rectangles,
                  depth-key bits, change votes), as one fixed IEEE float32
                  operation sequence, so both sides take those decisions in the
                  same precision (Sec. 3.2 voting; Supp. "Local Optimization
                  Kernel" tile mask and per-tile depth order).
  * sh          - real spherical harmonics up to degree 3 (colour model of the
                  base 3DGS method that Supp. "Implementation Details" adopts).
  * projection  - float64 EWA projection of 3D Gaussians to 2D conics.
  * composite   - float64 front-to-back alpha compositing, one pixel at a time
                  over the Gaussians whose 3-sigma tile rectangle holds the
                  pixel's tile, in (depth, index) order.
  * step        - the full-image loss, its exact gradient (autograd in float64)
                  restricted to the active set O^t (Sec. 3.3 "Local Optimization
                  Kernel": the local kernel must reproduce these gradients), and
                  the masked Adam step (Supp. "3DGS Optimization in Changed
                  Regions").
  * adam        - textbook Adam (Kingma & Ba) in float64.

Every function is pinned by `-m "not gpu"` tests against closed forms, library
special cases, brute force on tiny inputs and central finite differences.
"""
