"""GB300 (sm_103a) TV-L1 optical flow: the preconditioned dual solvers (pADMM, rpADMMI,
rpADMMII, Zach-pADMM, pDR) of Sun, Tai & Yuan (arXiv 2011.10979) inside a coarse-to-fine
pyramid, as hand-written CUDA kernels behind a C ABI (include/tvl1flow.h).

`flow` is the ctypes binding (same names as the C ABI), `build` compiles the library in-tree,
`synth` generates the seeded synthetic image pairs."""
