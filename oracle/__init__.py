"""FP64 CPU oracle for the MLS^2MC likelihood path (Latz, Papaioannou, Ullmann, arXiv:1709.09763).

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously correct
restatement of what the GPU library computes, used to check it. Only the tests,
the smoke check and the benchmark's CPU-baseline leg import it; the product
library (the CUDA path and its Python binding) never imports, links or runs it,
and it shares no code with that path.

Modules:
  kl       truncated KL table of the prior field (Sec. 5, Eq. truncKL)
  fem      P1 finite elements on the uniform triangulation (Sec. 5)
  forward  G_l(theta) and the Gaussian potential Phi (Sec. 2.1, Eq. phi)
  smc      cv/ESS, adaptive increments, evidence, resampling, pCN, MLS^2MC (Secs. 2-4)
  philox   Philox4x32-10 (Salmon et al. 2011) and the sampler's draw layout
  mlp      surrogate network forward/backward and Adam in FP64
  gaussian closed-form linear-Gaussian posterior and evidence (test reference)
"""
