"""CPU FP64 oracle for the dense-field phase-to-space (DF-P2S) turbulence simulator.

TEST INFRASTRUCTURE ONLY. This package is the slow, plain, obviously-correct
reference that the CUDA path is checked against. Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it. The product library never calls it, and it
shares no code, constants or tables with the CUDA sources.

Every function cites the part of the paper (Chimitt, Zhang, Mao, Chan,
"Real-Time Dense Field Phase-to-Space Simulation of Imaging through Atmospheric
Turbulence", arXiv 2210.06713) that it follows. Where the paper is silent the
reading taken is named in the docstring (R1..R31, the readings listed in the
design notes).

Modules
  zernike   Noll indexing, Zernike polynomials, Noll covariance A_0 (Sec. II-B)
  spectrum  path-integrated Zernike auto/cross spectra, lambda_j on the torus
            (Sec. III-A, III-C; R1, R2, R4, R5)
  noise     Philox-4x32-10 words and the Box-Muller Gaussians (R7, R8)
  sampler   FFT field sampler (Sec. III-A/III-C), dense-root variant, brute-force
            full-tensor sampler (Fig. rand_gen)
  fullsampler  the exact FFT sampler of the full cross-spectral density
            (Sec. III-B, no approximation; R29)
  p2s       pupil -> PSF (Eq. 2), SVD basis, projection weights (Sec. II-C)
  image     tilt warp and basis blur (Eq. 1, Eq. varying blur)
  mlp       the P2S surrogate network, forward/backward/Adam in FP64
  frame     the whole frame, step by step
  stats     lagged covariances of fields and their expectation A~(s) (Sec. III-D)
  aperture  structure function, LE / SE OTFs, tilt correlation and DTV of
            sampled fields (Sec. IV-B; R30)
  subharmonics  low-frequency compensation of the FFT sampler (Sec. IV-B; R31)
"""
