"""GB300-native DFEM S_n transport sweep (Tano & Ragusa, arXiv:1906.04017).

The compute path is the C-ABI library ``libsn_gb300.so`` (CUDA, sm_103a); this
package is its thin ctypes binding (``paper_1906_04017_gb300.sn``) and the
seeded workload generators (``paper_1906_04017_gb300.workloads``).
"""
