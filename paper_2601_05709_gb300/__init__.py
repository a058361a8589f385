"""GB300 (sm_103a) level-set shape optimisation with distributed shape derivatives.

The hot path of arXiv 2601.05709 (one iteration of its Algorithm 1 on a P1 Kuhn mesh) runs
in hand-written CUDA kernels behind the C ABI of include/formopt_gb300.h; ``api`` is the
Python binding of that ABI, ``workloads`` the seeded synthetic inputs.  Importing the
package does not load the library; ``api`` loads it on first use and fails loudly when it
has not been built.
"""
__all__ = ["api", "build", "workloads"]
