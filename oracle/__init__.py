"""CPU oracle for the constrained mobility-resistance solve.

TEST INFRASTRUCTURE ONLY.  Plain, slow, FP64 numpy code written from the
paper's equations, used to check the CUDA library.  Only the tests, the smoke
check and the CPU-baseline leg of the benchmark may import it; the product
(the C-ABI library and its Python binding) never does.

Modules:
  kinematics  quaternions and rotations (Sec. 2.1, App. B)
  mobility    RPY blob mobility, free space and no-slip wall (Sec. 2.3)
  system      K, C, B, the saddle-point operator A, its dense solution, the
              block-diagonal preconditioner and GMRES (Sec. 2.2-3.1)
  timestep    explicit Euler step with reconstruction and nonlinear
              correction (Sec. 4)
  wall_image  generated by gen_wall_image.py (regularised Blake image part)
"""
