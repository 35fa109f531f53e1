"""Test-infrastructure oracle for ABIP: a plain FP64 CPU implementation written from the
paper, and a brute-force LP solver for tiny instances.  Never imported by the product
package; only tests/, the smoke check and the benchmark's CPU-baseline leg use it."""
