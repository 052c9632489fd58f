"""FP64 CPU oracle for the colour-gradient lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, links or executes anything in this package; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code, tables or constants with the CUDA
path: every lattice constant below is restated here from the paper.

Layout
------
``lattice``    D3Q19 / D3Q7 velocity sets and weights, the eighth-order solid-
               normal stencil (Sec. 2.1, Eq. d3q19_weight_function,
               Eq. eigth_order_weight_function).
``cglbm``      the time step as separate whole-lattice passes, in the order of
               Sec. 2 and Appendix A (streaming, moments, colour field, wetting,
               curvature, exact-difference forcing, central-moment collision,
               recolouring, reaction, advection-diffusion), plus observables
               (Sec. 5.1).
``pointwise``  a deliberately naive per-node re-implementation (pure Python
               loops, recomputing every neighbour quantity from scratch) used to
               cross-check ``cglbm`` on tiny boxes and to evaluate sampled nodes
               of full-size lattices.

Parity status: every function is pinned by the ``-m "not gpu"`` tests
(conservation laws, the printed back-transformation rows, Poiseuille, Laplace,
contact angle, Gaussian diffusion, wall-reaction decay, reaction balance and the
pointwise cross-check).  Long-horizon bubble dynamics are chaotic and are
compared through observables only.
"""
