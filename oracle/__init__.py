"""CPU oracle for the skeleton executor — TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct CPU implementation of what the executor's
hot path computes, written from the paper (Soldado, Alexandre, Paulino,
"Execution of Compound Multi-Kernel OpenCL Computations in
Multi-CPU/Multi-GPU Environments"):

* ``oracle.image``    — the image stages (noise, solarise, mirror, 5x5 box
                        blur, 3-class threshold, class counts) and the
                        Filter Pipeline composition (Section 4 benchmarks);
* ``oracle.skeleton`` — depth-first evaluation of a skeleton computational
                        tree (Section 2, single-device execution model);
* ``oracle.nbody``    — FP64 direct-sum N-body with kick-drift-kick leapfrog
                        (Section 4, N-Body on the Loop skeleton), in plain C;
* ``oracle.mlp``      — FP64 forward/backward/Adam of the cost-model MLP
                        (no counterpart in the paper; it stands in for the
                        configuration-derivation step of Section 3.2);
* ``oracle.partition``— the partitioning constraints of Section 3.1;
* ``oracle.fft``      — forward and inverse DFT of every row, stage after
                        stage (Section 4, FFT pipelined with its inversion);
* ``oracle.batch``    — per-instance digests of a whole batch of Filter
                        Pipeline + blur instances, in a pool of processes.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or run anything here. The CUDA product path never
does, and shares no code with it: the two meet only through the seeded
generators in ``paper_1510_06585_gb300.inputs``.

Parity status per function is stated in each module's header.
"""
